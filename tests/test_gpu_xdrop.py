"""The x-drop (pre, post) form of the overlaps (Sec. 4.4) on the GPU against
the oracle, element by element and bit-exact: branch mask, chains, ranks,
orientations, contig offsets and bases, in the ASCII and the 2-bit outputs.

Inputs: the paper's worked example and two hand-derived variants; generated
graphs whose overlaps are reported with equal or unequal early starts; the
same graphs with uniformly random (pre, post), where many pieces are empty;
closed chains; batches; and the 100 Mb genome graph.
"""
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


def random_xdrop(G, seed):
    """Uniform (pre, post) in range for every entry: reads' reported overlaps
    cross freely, so many pieces are empty."""
    rng = np.random.default_rng(seed)
    rp = np.asarray(G.row_ptr, np.int64)
    u = np.repeat(np.arange(len(G.len)), np.diff(rp))
    lu, lv = np.asarray(G.len)[u], np.asarray(G.len)[np.asarray(G.col)]
    X = gen.with_xdrop(G)
    X.pre = np.floor(rng.random(len(u)) * lu).astype(np.int32)
    X.post = np.floor(rng.random(len(u)) * lv).astype(np.int32)
    return X


def check(ctx, G, mcr=2, **kw):
    orc = oracle.run(G, min_chain_reads=mcr)
    gpu = run_gpu(ctx, G, min_chain_reads=mcr, **kw)
    assert_parity(gpu, orc)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    try:
        off2, packed, total = cg.contigs_2bit_host(g)
    finally:
        g.close()
    assert np.array_equal(off2, orc.contig_off)
    want = np.zeros(cg.packed_bytes_2bit(orc.total_bases), np.uint8)
    p2 = oracle.pack2(orc.bases)
    want[: p2.size] = p2
    assert np.array_equal(packed, want)
    return orc


def test_paper_examples(ctx):
    for name, c in _pins._xdrop_cases().items():
        for stored1_rc in (False, True):
            G = _pins.xdrop_chain(c["reads"], c["pp"], stored1_rc)
            for mcr in (1, 3):
                orc = check(ctx, G, mcr)
                assert orc.contig(0).decode() == c["contig"], name


@pytest.mark.parametrize("consistent", [True, False])
def test_generated_with_trims(ctx, consistent):
    G = gen.generate("tiny-1Mb", threads=8, off_align=1)
    for trim, seed in ((0, 0), (40, 1), (5000, 2)):
        X = gen.with_xdrop(G, max_trim=trim, seed=seed, consistent=consistent)
        orc = check(ctx, X, 2)
        if consistent:
            assert np.array_equal(orc.bases, oracle.run(G, min_chain_reads=2).bases)


def test_random_coordinates_and_empty_pieces(ctx):
    G = gen.generate("tiny-1Mb", threads=8, off_align=4)
    for seed in range(3):
        X = random_xdrop(G, seed)
        check(ctx, X, 1)
        check(ctx, X, 2, inputs="device", outputs="device")


def test_closed_and_long_chains(ctx):
    sizes = [20_000, 3, 4, 5, 7, 16, 33, 100] + [2] * 300 + [1] * 50
    closed = [False] + [True] * 7 + [False] * 350
    G = structured(6, sizes, closed, lone=40, align=1)
    for mcr in (1, 2):
        check(ctx, gen.with_xdrop(G, max_trim=10, seed=5, consistent=False), mcr)
        check(ctx, random_xdrop(G, 7), mcr)
    for seed in (4, 9):
        C = _pins.circular_graph(seed, 900, 120, 45)
        check(ctx, gen.with_xdrop(C, max_trim=30, seed=seed), 1)


def test_batch_of_xdrop_graphs(ctx):
    graphs = [gen.with_xdrop(gen.generate(gen.batched_graph(j), threads=8), max_trim=60, seed=j, consistent=False)
              for j in (0, 3, 17)]
    want = [oracle.run(X, min_chain_reads=2) for X in graphs]
    g = cg.cg_load_batch(ctx, graphs)
    try:
        off, bases = cg.contigs_host(g)
        fc, fb = cg.cg_batch_ranges(g)
    finally:
        g.close()
    for j, w in enumerate(want):
        assert np.array_equal(off[fc[j]:fc[j + 1] + 1] - fb[j], w.contig_off)
        assert np.array_equal(bases[fb[j]:fb[j + 1]], w.bases)
    # a batch mixes no forms
    with pytest.raises(cg.CgError) as e:
        cg.cg_load_batch(ctx, [graphs[0], gen.generate(gen.batched_graph(3), threads=8)])
    assert e.value.status == cg.CG_EINVAL


def test_invalid_coordinates_rejected(ctx):
    c = _pins._xdrop_cases()["paper"]
    for field, i, val in (("pre", 0, 6), ("pre", 0, -1), ("post", 2, 7), ("post", 1, -1)):
        G = _pins.xdrop_chain(c["reads"], c["pp"], False)
        getattr(G, field)[i] = val
        assert not oracle.validate(G)[0]
        with pytest.raises(cg.CgError) as e:
            cg.cg_load_graph(ctx, G)
        assert e.value.status == cg.CG_EGRAPH
    G = _pins.xdrop_chain(c["reads"], c["pp"], False)
    G.pre[2] = 7                                   # in range for u = l1 although l2 is shorter
    check(ctx, G, 1)


def test_genome_100mb(ctx):
    G = gen.generate("genome-100Mb", threads=16)
    check(ctx, gen.with_xdrop(G, max_trim=200, seed=11, consistent=False), 2)
