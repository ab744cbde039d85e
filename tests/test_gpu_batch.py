"""Batched form against the plain form and the oracle: graphs loaded as one
union graph give, slice by slice, exactly each graph's own contigs."""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg
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


def _check_batch(ctx, graphs, mcr):
    g = cg.cg_load_batch(ctx, graphs, min_chain_reads=mcr)
    try:
        cid, rank, orient, n_contigs, n_cycles = cg.chains_host(g)
        off, bases = cg.contigs_host(g)
        first_contig, first_base = cg.cg_batch_ranges(g)
    finally:
        g.close()
    assert first_contig[0] == 0 and first_base[0] == 0
    assert first_contig[-1] == n_contigs and first_base[-1] == len(bases)
    R = 0
    for j, G in enumerate(graphs):
        want = oracle.run(G, min_chain_reads=mcr)
        c0, c1 = int(first_contig[j]), int(first_contig[j + 1])
        assert c1 - c0 == want.n_contigs
        assert np.array_equal(off[c0:c1 + 1] - off[c0], want.contig_off)
        assert np.array_equal(bases[int(first_base[j]):int(first_base[j + 1])], want.bases)
        sl = slice(R, R + G.n)
        assert np.array_equal(np.where(cid[sl] >= 0, cid[sl] - R, -1), want.chain_id)
        assert np.array_equal(rank[sl], want.rank) and np.array_equal(orient[sl], want.orient)
        R += G.n


def test_batch_of_generated_graphs(ctx):
    graphs = [gen.generate(gen.batched_graph(j), threads=8) for j in range(24)]
    _check_batch(ctx, graphs, 2)
    _check_batch(ctx, graphs[:9], 1)


def test_batch_of_mixed_graphs(ctx):
    # different row_ptr widths are refused; equal widths with cycles, lone reads, empty graphs work
    graphs = [structured(s, [300, 4, 5, 2, 2, 1], [False, True, True, False, False, False], lone=7) for s in range(5)]
    graphs.append(structured(99, [1]))
    graphs += [gen.generate("tiny-1Mb", threads=8)]
    for G in graphs:
        G.row_ptr = G.row_ptr.astype(np.int64)
    _check_batch(ctx, graphs, 1)
    _check_batch(ctx, graphs, 2)
    with pytest.raises(cg.CgError):
        bad = [graphs[0], structured(3, [3])]
        bad[1].row_ptr = bad[1].row_ptr.astype(np.int32)
        cg.cg_load_batch(ctx, bad)


def test_batch_one_graph_equals_plain(ctx):
    G = gen.generate(gen.batched_graph(77), threads=8)
    b = cg.cg_load_batch(ctx, [G])
    p = cg.cg_load_graph(ctx, G)
    try:
        ob, bb = cg.contigs_host(b)
        op, bp = cg.contigs_host(p)
        assert np.array_equal(ob, op) and np.array_equal(bb, bp)
    finally:
        b.close()
        p.close()


def _pinned_at(a, offset, keep):
    """a's values in pinned host memory, `offset` bytes into a pinned buffer (so
    that the copy may start at any alignment)."""
    import torch
    buf = torch.empty(a.nbytes + offset + 16, dtype=torch.uint8, pin_memory=True)
    keep.append(buf)
    v = buf.numpy()[offset: offset + a.nbytes].view(a.dtype)
    v[...] = a
    return v


def test_batch_from_pinned_memory_in_place(ctx):
    """Every input array of every graph in pinned memory: the batch is read in
    place by the copy kernel, at 16-byte, 4-byte and byte alignments (arrays
    placed at offsets 0..7 into their buffers), with the reads in pinned
    memory too (copied into the union, or read in place with HOST_READS)."""
    keep = []
    graphs = [gen.generate(gen.batched_graph(j), threads=8) for j in range(12)]
    graphs.append(structured(5, [300, 4, 5, 2, 2, 1], [False, True, True, False, False, False], lone=7))
    graphs[-1].row_ptr = graphs[-1].row_ptr.astype(np.int32)
    want = [oracle.run(G, min_chain_reads=2) for G in graphs]
    pinned = []
    for j, G in enumerate(graphs):
        P = type("P", (), {})()
        for i, k in enumerate(("row_ptr", "col", "code", "suf", "len", "off")):
            setattr(P, k, _pinned_at(getattr(G, k), (j + 3 * i) % 8, keep))
        P.packed = _pinned_at(G.packed, 0, keep)           # HOST_READS wants the reads 4-byte aligned
        pinned.append(P)
    for flags in (0, cg.HOST_READS):
        g = cg.cg_load_batch(ctx, pinned, flags=flags, min_chain_reads=2)
        try:
            off, bases = cg.contigs_host(g)
            fc, fb = cg.cg_batch_ranges(g)
        finally:
            g.close()
        for j, w in enumerate(want):
            c0, c1 = int(fc[j]), int(fc[j + 1])
            assert c1 - c0 == w.n_contigs, j
            assert np.array_equal(off[c0:c1 + 1] - off[c0], w.contig_off), j
            assert np.array_equal(bases[int(fb[j]):int(fb[j + 1])], w.bases), j
