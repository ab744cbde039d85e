"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times (device-resident inputs borrowed in place, default tuning, stages
replayed from CUDA graphs; host-resident reads with in-place host outputs):

- the 3.1 Gb genome-shaped graph (6.2M reads, 23 GB of packed reads, 3.3 Gb
  of contigs): every contig offset and base against the oracle, which runs
  on the whole graph, plus the per-read chains and the 2-bit form; the same
  through CG_HOST_READS into pinned host buffers; the graph in the x-drop
  form (early starts up to 200 bases, unequal); the transitive reduction of
  the recipe's overlap graph before reduction (3.4M entries);
The batched and served workloads are in test_gpu_fullsize_forms.py.
"""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_04350_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    c = cg.cg_create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def genome():
    import torch
    keep = []

    def alloc(shape, dt):                       # pinned, as bench.py generates it
        t = torch.empty(shape, dtype=getattr(torch, dt.__name__), pin_memory=True)
        keep.append(t)
        return t.numpy()
    G = gen.generate("genome-3.1Gb", keep_genome=False, alloc=alloc)
    G._pinned = keep
    orc = oracle.run(G, min_chain_reads=2, validate=False)
    return G, orc


def assert_bases(got, want):
    if not np.array_equal(got, want):
        bad = int(np.nonzero(got != want)[0][0]) if got.size == want.size else -1
        raise AssertionError(f"bases differ (first at {bad}; sizes {got.size}, {want.size})")


def test_genome_3_1gb_full(ctx, genome):
    import torch
    G, orc = genome
    D = type("D", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(D, k, torch.from_numpy(getattr(G, k)).cuda())
    g = cg.cg_load_graph(ctx, D, flags=cg.BORROW_DEVICE, min_chain_reads=2)
    try:
        n_contigs, total = cg.cg_emit_contigs(g)
        assert (n_contigs, total) == (orc.n_contigs, orc.total_bases)
        off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
        bases = torch.empty((total + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
        cg.cg_emit_contigs(g, off, bases)
        cg.cg_sync(ctx)
        assert np.array_equal(off.cpu().numpy(), orc.contig_off)
        assert_bases(bases[:total].cpu().numpy(), orc.bases)
        del bases
        cid, rank, orient = (np.empty(G.n, np.int32), np.empty(G.n, np.int32), np.empty(G.n, np.uint8))
        cg.cg_chains(g, cid, rank, orient)
        assert np.array_equal(cid, orc.chain_id) and np.array_equal(rank, orc.rank)
        assert np.array_equal(orient, orc.orient)
        off2, packed, total2 = cg.contigs_2bit_host(g)
        assert total2 == total
        want = oracle.pack2(orc.bases)
        assert np.array_equal(packed[: want.size], want) and not packed[want.size:].any()
    finally:
        g.close()


def test_genome_3_1gb_host_reads(ctx, genome):
    import torch
    G, orc = genome
    g = cg.cg_load_graph(ctx, G, flags=cg.HOST_READS, min_chain_reads=2)
    try:
        off = torch.empty(orc.n_contigs + 1, dtype=torch.int64, pin_memory=True).numpy()
        bases = torch.empty(max(orc.total_bases, 16), dtype=torch.uint8, pin_memory=True).numpy()
        cg.cg_emit_contigs(g, off, bases)
        assert np.array_equal(off, orc.contig_off)
        assert_bases(bases[: orc.total_bases], orc.bases)
    finally:
        g.close()


def test_genome_3_1gb_xdrop(ctx, genome):
    G, _ = genome
    X = gen.with_xdrop(G, max_trim=200, seed=7, consistent=False)
    orc = oracle.run(X, min_chain_reads=2, validate=False)
    g = cg.cg_load_graph(ctx, X, min_chain_reads=2)
    try:
        off, bases = cg.contigs_host(g)
    finally:
        g.close()
    assert np.array_equal(off, orc.contig_off)
    assert_bases(bases, orc.bases)


def test_transitive_reduction_3_1gb(ctx):
    R = gen.generate(dict(gen.WORKLOADS["genome-3.1Gb"](), full_overlaps=1), keep_genome=False, with_packed=False)
    S = cg.cg_transitive_reduction(ctx, R)
    W = oracle.transitive_reduction(R)
    for k in ("row_ptr", "col", "code", "suf"):
        assert np.array_equal(np.asarray(getattr(S, k)).astype(np.int64), np.asarray(getattr(W, k)).astype(np.int64)), k
