"""CUDA path (through the C ABI) against the CPU oracle, element by element.

All outputs are integers or bytes, so the bar is bit-exact: the branch mask,
per-read chain id / rank / orientation, contig offsets and every contig base.
Sizes span many scan tiles (2048 reads), emission tiles (8 KiB) and a ragged
tail; the named workloads are the tiny 1 Mb graph, the 100 Mb genome graph
(full compare) and the 3.1 Gb genome graph in the benchmark's configuration.
"""
import random

import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg
from tests import _pins
from tests._gpu import assert_parity, run_gpu
from tests._graphs import structured

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_04350_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    c = cg.cg_create(0)
    yield c
    c.close()


def check(ctx, G, mcr=2, **kw):
    orc = oracle.run(G, min_chain_reads=mcr)
    gpu = run_gpu(ctx, G, min_chain_reads=mcr, **kw)
    assert_parity(gpu, orc)
    return orc


def test_paper_examples(ctx):
    for stored_rc in (False, True):
        G, want = _pins._concat_graph(stored_rc)
        orc = check(ctx, G, 2)
        assert orc.contig(0).decode() == want
    rnd = random.Random(7)
    reads = ["".join(rnd.choice("ACGT") for _ in range(12)) for _ in range(8)]
    ent = []
    for u, v in [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (2, 6), (6, 7)]:
        ent += [(u, v, 1, 5), (v, u, 2, 4)]
    for mcr in (1, 2):
        check(ctx, _pins.graph_from(reads, ent), mcr)


def test_brute_force_graphs(ctx):
    rnd = random.Random(2024)
    for t in range(150):
        if t % 2 == 0:
            G = _pins.random_tiny_graph(rnd, rnd.randint(1, 8), rnd.choice([0.15, 0.3, 0.5]))
        else:
            G = _pins.random_chain_graph(rnd, rnd.randint(1, 12), rnd.randint(0, 3))
        check(ctx, G, rnd.choice([1, 2, 3]))


@pytest.mark.parametrize("align", [1, 4, 32])
@pytest.mark.parametrize("mcr", [1, 2])
def test_tiny_1mb(ctx, align, mcr):
    G = gen.generate("tiny-1Mb", threads=8, off_align=align)
    check(ctx, G, mcr)


@pytest.mark.parametrize("rp_bytes", [4, 8])
@pytest.mark.parametrize("mcr", [1, 2])
def test_borrowed_row_ptr_not_16_byte_aligned(ctx, rp_bytes, mcr):
    """A borrowed row_ptr that starts 4 or 8 bytes past a 16-byte boundary is
    read without vector loads; the 1 Mb graph spans several 128-read passes
    of the mask stage and a ragged tail."""
    import torch
    from types import SimpleNamespace
    G = gen.generate("tiny-1Mb", threads=8, rp_bytes=rp_bytes)
    orc = oracle.run(G, min_chain_reads=mcr)
    rp = np.asarray(G.row_ptr)
    padded = torch.zeros(rp.shape[0] + 1, dtype=torch.int64 if rp_bytes == 8 else torch.int32, device="cuda")
    padded[1:] = torch.from_numpy(rp).cuda()
    src = SimpleNamespace(row_ptr=padded[1:], **{k: torch.from_numpy(np.ascontiguousarray(getattr(G, k))).cuda()
                                                 for k in ("col", "code", "suf", "len", "off", "packed")})
    assert src.row_ptr.data_ptr() % 16 != 0
    g = cg.cg_load_graph(ctx, src, flags=cg.BORROW_DEVICE, min_chain_reads=mcr)
    try:
        isb = np.empty(G.n, np.uint8)
        assert cg.cg_mask_branches(g, isb) == orc.n_branch
        assert np.array_equal(isb, orc.is_branch)
        cid, rank, orient, nc, ncy = cg.chains_host(g)
        assert np.array_equal(cid, orc.chain_id) and np.array_equal(rank, orc.rank)
        off, bases = cg.contigs_host(g)
        assert np.array_equal(off, orc.contig_off) and np.array_equal(bases, orc.bases)
    finally:
        g.close()


def test_device_inputs_and_outputs(ctx):
    G = gen.generate("tiny-1Mb", threads=8)
    orc = oracle.run(G, min_chain_reads=2)
    for inputs, outputs, flags in [("device", "device", 0), ("device", "host", cg.BORROW_DEVICE),
                                   ("host", "device", 0), ("device", "device", cg.BORROW_DEVICE | cg.NO_VALIDATE)]:
        assert_parity(run_gpu(ctx, G, 2, inputs=inputs, outputs=outputs, flags=flags), orc)


def test_long_chains_and_cycles(ctx):
    # one 200k-read chain (deep list ranking), closed chains of many lengths,
    # lone reads, short chains; spans ~100 scan tiles and many emission tiles
    sizes = [200_000] + [3, 4, 5, 7, 16, 33, 100, 1000, 5000] + [2] * 500 + [1] * 300 + list(range(2, 60))
    closed = [False] + [True] * 9 + [False] * (500 + 300 + 58)
    G = structured(5, sizes, closed, lone=200, align=1)
    for mcr in (1, 2, 3):
        check(ctx, G, mcr)


def test_only_cycles_and_ruler_free_cycles(ctx):
    sizes = [3] * 300 + [4] * 200 + [9] * 50 + [40] * 20 + [3000]
    G = structured(9, sizes, [True] * len(sizes), align=4)
    orc = check(ctx, G, 2)
    assert orc.n_cycles == len(sizes)


def test_degenerate_graphs(ctx):
    # no reads at all
    empty = structured(3, [], lone=0)
    assert empty.n == 0
    orc = check(ctx, empty, 2)
    assert orc.n_contigs == 0 and orc.total_bases == 0
    # a single read, no overlaps at all, everything masked
    one = structured(1, [1])
    check(ctx, one, 1)
    check(ctx, one, 2)
    lone = structured(2, [1] * 5000)
    check(ctx, lone, 1)
    check(ctx, lone, 2)
    rnd = random.Random(3)
    reads = ["".join(rnd.choice("ACGT") for _ in range(10)) for _ in range(4)]
    star = [(0, k, 1, 5) for k in (1, 2, 3)] + [(k, 0, 2, 5) for k in (1, 2, 3)]
    check(ctx, _pins.graph_from(reads, star), 1)
    bigdeg = _pins.random_tiny_graph(rnd, 12, 0.9)
    check(ctx, bigdeg, 1)


def test_generated_small_sweep(ctx):
    for seed in range(6):
        d = gen._cfg(1000 + seed, 2_000_000, [(0.06, 2000, 9000, 2, 12, 0.0)], 25, 1, 8000, 4000, 2500)
        G = gen.generate(d, threads=8, off_align=(1, 4, 32)[seed % 3])
        check(ctx, G, 1 + seed % 2)


def test_batched_pool_graphs(ctx):
    for j in (0, 7, 100, 511):
        check(ctx, gen.generate(gen.batched_graph(j), threads=8), 2)


def test_genome_100mb_full(ctx):
    G = gen.generate("genome-100Mb", threads=16)
    for mcr in (2, 1):
        check(ctx, G, mcr)


def test_invalid_graphs_rejected(ctx):
    G, _ = _pins._concat_graph(False)
    bad = []
    for field, idx, val in [("code", 1, 0), ("col", 0, 7), ("col", 0, 0), ("suf", 0, 0), ("suf", 0, 8),
                            ("code", 0, 4), ("off", 2, 10**6), ("off", 0, -1), ("len", 0, 0), ("row_ptr", 1, 5)]:
        H = _pins.graph_from(G.reads, [])
        for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
            setattr(H, k, getattr(G, k).copy())
        getattr(H, field)[idx] = val
        bad.append(H)
    bad.append(_pins.graph_from(G.reads, [(0, 1, 1, 4), (0, 1, 1, 3), (1, 0, 2, 2), (1, 2, 1, 2), (2, 1, 2, 5)]))
    bad.append(_pins.graph_from(G.reads, [(0, 1, 1, 4), (1, 0, 2, 2), (1, 2, 1, 2)]))
    bad.append(_pins.graph_from(G.reads[:1], [(0, 0, 3, 2)]))   # a self overlap, nothing else wrong
    # one well-formed entry more than row_ptr[n] counts
    H = _pins.graph_from(G.reads, [])
    for k in ("row_ptr", "len", "off", "packed"):
        setattr(H, k, getattr(G, k).copy())
    H.col, H.code, H.suf = (np.append(a, a[0]).astype(a.dtype) for a in (G.col, G.code, G.suf))
    bad.append(H)
    # the last read one base past the packed stream's end
    end = len(G.packed) * 4
    H = _pins.graph_from(G.reads, [])
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(H, k, getattr(G, k).copy())
    H.off[2] = end - int(G.len[2]) + 1
    bad.append(H)
    for H in bad:
        assert not oracle.validate(H)[0]
        with pytest.raises(cg.CgError) as e:
            cg.cg_load_graph(ctx, H)
        assert e.value.status == cg.CG_EGRAPH
    # the context is still usable afterwards
    check(ctx, G, 2)
    # a read that ends on the stream's last base is in bounds, on both sides
    H.off[2] = end - int(G.len[2])
    assert oracle.validate(H)[0]
    check(ctx, H, 2)


def test_small_capacity_rejected(ctx):
    G = gen.generate("tiny-1Mb", threads=8)
    g = cg.cg_load_graph(ctx, G)
    n_contigs, total = cg.cg_emit_contigs(g)
    with pytest.raises(cg.CgError) as e:
        cg.cg_emit_contigs(g, np.empty(n_contigs + 1, np.int64), np.empty(total - 1, np.uint8))
    assert e.value.status == cg.CG_EINVAL
    import torch
    small = torch.empty(total - 16, dtype=torch.uint8, device="cuda")
    cg.cg_emit_contigs(g, None, small, want_counts=False)
    with pytest.raises(cg.CgError) as e:
        cg.cg_sync(ctx)
    assert e.value.status == cg.CG_EINVAL
    # device contig offsets one entry short, spelled in the same replayed stage as
    # the bases: the piece scan writes none of them and the next wait reports it
    full = torch.empty((total + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
    short = torch.full((n_contigs,), -5, dtype=torch.int64, device="cuda")
    cg.cg_emit_contigs(g, short, full, want_counts=False)
    with pytest.raises(cg.CgError) as e:
        cg.cg_sync(ctx)
    assert e.value.status == cg.CG_EINVAL
    assert (short.cpu().numpy() == -5).all()
    off_d = torch.full((n_contigs + 1,), -5, dtype=torch.int64, device="cuda")
    cg.cg_emit_contigs(g, off_d, full, want_counts=False)
    cg.cg_sync(ctx)
    off, bases = cg.contigs_host(g)          # still usable
    g.close()
    orc = oracle.run(G)
    assert np.array_equal(bases, orc.bases)
    assert np.array_equal(off_d.cpu().numpy(), orc.contig_off)


@pytest.mark.parametrize("ruler_log2,tile_bytes,bps,bt", [(1, 4096, 1, 256), (2, 8192, 2, 128), (4, 16384, 8, 512),
                                                          (7, 32768, 4, 128), (12, 32768, 3, 256), (3, 65536, 8, 256),
                                                          (5, 131072, 6, 512), (3, 32768, 16, 128), (3, 32768, 2, 512)])
def test_tuning_does_not_change_output(ruler_log2, tile_bytes, bps, bt):
    """Launch parameters chosen by the autotuner never change a byte."""
    c = cg.cg_create(0)
    try:
        cg.cg_set_tuning(c, ruler_log2=ruler_log2, tile_bytes=tile_bytes, emit_blocks_per_sm=bps, emit_block_threads=bt)
        assert cg.cg_get_tuning(c) == {"ruler_log2": ruler_log2, "tile_bytes": tile_bytes, "emit_blocks_per_sm": bps,
                                       "emit_block_threads": bt}
        check(c, structured(21, [50_000, 3, 4, 17] + [2] * 40 + [6] * 30, [False, True, True, True] + [False] * 70,
                            lone=50, align=1), 1)
        check(c, gen.generate(gen.batched_graph(11), threads=8), 2)
    finally:
        c.close()


@pytest.mark.parametrize("pdl", [False, True])
def test_graphs_off_and_replay_with_new_buffers(pdl):
    """Stages launched one by one give the same bytes as replayed CUDA graphs,
    with or without programmatic dependent launch, also when the output
    buffers change between replays."""
    import torch
    G = structured(31, [20_000, 5, 9] + [2] * 300 + [7] * 50, [False, True, True] + [False] * 350, lone=100)
    orc = oracle.run(G, min_chain_reads=1)
    for graphs in (False, True):
        c = cg.cg_create(0)
        try:
            cg.cg_set_graphs(c, graphs)
            cg.cg_set_pdl(c, pdl)
            assert_parity(run_gpu(c, G, 1), orc)
            g = cg.cg_load_graph(c, G, min_chain_reads=1)
            n_contigs, total = cg.cg_emit_contigs(g)
            for rep in range(3):
                off = torch.empty(n_contigs + 1 + rep, dtype=torch.int64, device="cuda")
                bases = torch.empty(total + 16 * rep + 16, dtype=torch.uint8, device="cuda")
                cg.cg_mask_branches(g, want_count=False)
                cg.cg_chains(g, want_counts=False)
                cg.cg_emit_contigs(g, off, bases, want_counts=False)
                cg.cg_sync(c)
                assert np.array_equal(off.cpu().numpy()[:n_contigs + 1], orc.contig_off)
                assert np.array_equal(bases.cpu().numpy()[:total], orc.bases)
            g.close()
        finally:
            c.close()


@pytest.mark.parametrize("graphs,pdl,timing", [(False, True, 0), (True, False, 0), (True, True, 0), (True, True, 1),
                                               (True, True, 2), (True, True, 3), (False, True, 2)])
def test_launch_modes_repeat_identically(graphs, pdl, timing):
    """Every launch mode (graphs, programmatic dependent launch, timing events
    between kernels or around the spelling) gives the oracle's bytes, and
    twenty back-to-back device-output runs of one graph stay identical."""
    import torch
    G = gen.generate("tiny-1Mb", threads=8)
    orc = oracle.run(G)
    c = cg.cg_create(0)
    try:
        cg.cg_set_graphs(c, graphs)
        cg.cg_set_pdl(c, pdl)
        cg.cg_set_timing(c, timing)
        g = cg.cg_load_graph(c, G)
        n_contigs, total = cg.cg_emit_contigs(g)
        assert n_contigs == orc.n_contigs
        off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
        bases = torch.empty((total + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
        outs = []
        for rep in range(20):
            cg.cg_mask_branches(g, want_count=False)
            cg.cg_chains(g, want_counts=False)
            cg.cg_emit_contigs(g, off, bases, want_counts=False)
            if rep % 5 == 4:
                outs.append((off.clone(), bases.clone()))
        cg.cg_sync(c)
        for o, b in outs:
            assert np.array_equal(o.cpu().numpy(), orc.contig_off)
            assert np.array_equal(b.cpu().numpy()[:total], orc.bases)
        g.close()
    finally:
        c.close()


def test_repeat_runs_are_identical(ctx):
    G = gen.generate(gen.batched_graph(3), threads=8)
    g = cg.cg_load_graph(ctx, G)
    first = cg.contigs_host(g)
    for _ in range(5):
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        off, bases = cg.contigs_host(g)
        assert np.array_equal(off, first[0]) and np.array_equal(bases, first[1])
    g.close()
