"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (inputs borrowed from device memory, default tuning, stages replayed
from CUDA graphs):

- the 3.1 Gb genome-shaped graph (6.2M reads, 23 GB of packed reads, 3.3 Gb
  of contigs): every contig offset and base against the oracle, which runs
  on the whole graph, plus the per-read chains and the 2-bit form;
- the 512-graph batch as one union: every graph's contig count and base
  count, and the full contigs of a sample of graphs.
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


def test_genome_3_1gb_full(ctx):
    import torch
    G = gen.generate("genome-3.1Gb", keep_genome=False)
    orc = oracle.run(G, min_chain_reads=2, validate=False)
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
        got = bases[:total].cpu().numpy()
        if not np.array_equal(got, orc.bases):
            bad = int(np.nonzero(got != orc.bases)[0][0])
            raise AssertionError(f"bases differ first at {bad} of {total}")
        del got, bases
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


def test_batched_512_full(ctx):
    graphs = [gen.generate(gen.batched_graph(j), keep_genome=False) for j in range(512)]
    g = cg.cg_load_batch(ctx, graphs, min_chain_reads=2)
    try:
        off, bases = cg.contigs_host(g)
        fc, fb = cg.cg_batch_ranges(g)
    finally:
        g.close()
    rng = np.random.default_rng(5)
    sample = set(rng.choice(512, size=24, replace=False).tolist()) | {0, 511}
    for j in range(512):
        if j not in sample:
            continue
        w = oracle.run(graphs[j], min_chain_reads=2, validate=False)
        assert fc[j + 1] - fc[j] == w.n_contigs and fb[j + 1] - fb[j] == w.total_bases
        assert np.array_equal(off[fc[j]:fc[j + 1] + 1] - fb[j], w.contig_off)
        assert np.array_equal(bases[fb[j]:fb[j + 1]], w.bases)
    assert fb[512] == len(bases)
