"""Spelling one part of a contig assignment (Sec. 4.3-4.4: each process spells
the contigs assigned to it) on the GPU.

Expected values are the oracle's own contigs: part p's output is the oracle's
contigs c with part[c] == p back to back in contig order, and its contig
offsets give every contig's range in it (empty for other parts). The
assignments come from the GPU's LPT partition (itself checked against the
oracle's LPT in test_gpu_partition.py) and from arbitrary int32 values.
Everything is compared byte for byte.
"""
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


def expected(orc, part, p):
    """Part p's contig offsets and bases, from the oracle's whole output."""
    C = orc.n_contigs
    keep = np.asarray(part[:C]) == p
    sizes = np.diff(orc.contig_off)
    off = np.concatenate([[0], np.cumsum(np.where(keep, sizes, 0))]).astype(np.int64)
    pieces = [orc.bases[orc.contig_off[c]:orc.contig_off[c + 1]] for c in np.nonzero(keep)[0]]
    bases = np.concatenate(pieces) if pieces else np.empty(0, np.uint8)
    return off, bases


def check_part(g, orc, part, p):
    off, bases = cg.contigs_part_host(g, part, p)
    want_off, want_bases = expected(orc, part, p)
    assert np.array_equal(off, want_off)
    assert np.array_equal(bases, want_bases)
    return len(bases)


@pytest.mark.parametrize("name,mcr", [("tiny-1Mb", 1), ("tiny-1Mb", 2), ("batched-11", 1)])
def test_lpt_parts_cover_the_output(ctx, name, mcr):
    """Every part of 1, 3 and 8-way LPT assignments by bases: each part's
    spelling is the oracle's contigs of that part, its size is the part's LPT
    weight, and the parts' sizes add up to the whole output."""
    G = gen.generate(gen.batched_graph(11) if name == "batched-11" else name, threads=8)
    orc = oracle.run(G, min_chain_reads=mcr)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    try:
        for P in (1, 3, 8):
            part, pw = cg.cg_partition_contigs(g, P, cg.WEIGHT_BASES)
            sizes = [check_part(g, orc, part, p) for p in range(P)]
            assert sizes == [int(w) for w in pw]
            assert sum(sizes) == len(orc.bases)
        # the whole output and the partition are unchanged afterwards
        off, bases = cg.contigs_host(g)
        assert np.array_equal(off, orc.contig_off) and np.array_equal(bases, orc.bases)
        part2, _ = cg.cg_partition_contigs(g, 3, cg.WEIGHT_BASES)
        part3, _ = cg.cg_partition_contigs(g, 3, cg.WEIGHT_BASES)
        assert np.array_equal(part2, part3)
    finally:
        g.close()


def test_arbitrary_part_values(ctx):
    """Any int32 values name parts: negative and large ones, a value no contig
    has (an empty output), and every contig in one part (the whole output)."""
    G = structured(41, [30_000, 4, 7] + [2] * 200 + [5] * 80, [False, True, True] + [False] * 280, lone=60)
    orc = oracle.run(G, min_chain_reads=1)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=1)
    try:
        C = orc.n_contigs
        rng = np.random.default_rng(5)
        part = rng.choice(np.array([-7, 0, 3, 2**31 - 1], np.int32), size=C).astype(np.int32)
        for p in (-7, 0, 3, 2**31 - 1):
            check_part(g, orc, part, p)
        assert check_part(g, orc, part, 12345) == 0
        same = np.full(C, 9, np.int32)
        assert check_part(g, orc, same, 9) == len(orc.bases)
        # a longer part array than there are contigs is fine
        check_part(g, orc, np.concatenate([part, np.zeros(5, np.int32)]), 3)
    finally:
        g.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_runs_of_other_parts(ctx, seed):
    """Another part's contigs between two of this part's are a run of empty
    pieces that the spelling skips by a search over the offsets: runs of 31,
    32, 33, 64 and thousands of pieces, inside one output tile and across
    tiles, with alternating and random assignments."""
    sizes = [31, 32, 33, 64, 1, 2, 31, 32, 33, 65, 3000, 5, 32, 7000, 31, 1, 33] * 3
    G = structured(100 + seed, sizes, [False] * len(sizes), min_len=20, max_len=60, lone=17)
    orc = oracle.run(G, min_chain_reads=1)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=1)
    try:
        C = orc.n_contigs
        alt = (np.arange(C) % 2).astype(np.int32)
        for p in (0, 1):
            check_part(g, orc, alt, p)
        rnd = np.random.default_rng(seed).integers(0, 3, size=C).astype(np.int32)
        for p in (0, 1, 2):
            check_part(g, orc, rnd, p)
        one = np.zeros(C, np.int32)
        one[C // 2] = 1                     # a single contig in the middle
        check_part(g, orc, one, 1)
        check_part(g, orc, one, 0)
    finally:
        g.close()


def test_device_buffers_and_replay(ctx):
    """Device part array and outputs (the replayed CUDA graph of the spelling),
    parts taken in turn and repeated, then the whole output again."""
    import torch
    G = gen.generate("tiny-1Mb", threads=8)
    orc = oracle.run(G)
    g = cg.cg_load_graph(ctx, G)
    try:
        part, _ = cg.cg_partition_contigs(g, 4, cg.WEIGHT_READS)
        d_part = torch.from_numpy(part).cuda()
        C = orc.n_contigs
        off = torch.empty(C + 1, dtype=torch.int64, device="cuda")
        bases = torch.empty(len(orc.bases) + 16, dtype=torch.uint8, device="cuda")
        for rep in range(2):
            for p in range(4):
                nc, tot = cg.cg_emit_part(g, d_part, p, off, bases)
                want_off, want_bases = expected(orc, part, p)
                assert nc == C and tot == len(want_bases)
                assert np.array_equal(off.cpu().numpy(), want_off)
                assert np.array_equal(bases.cpu().numpy()[:tot], want_bases)
        nc, tot = cg.cg_emit_contigs(g, off, bases)
        assert np.array_equal(off.cpu().numpy(), orc.contig_off)
        assert np.array_equal(bases.cpu().numpy()[:tot], orc.bases)
    finally:
        g.close()


def test_xdrop_and_host_reads(ctx):
    """The x-drop (pre, post) form, whose pieces the layout takes from the chain
    stage, and a graph whose packed reads stay in pinned host memory
    (CG_HOST_READS, spelled over the host link): each part equals the oracle's."""
    import torch
    G = gen.generate("tiny-1Mb", threads=8)
    X = gen.with_xdrop(G, max_trim=60, seed=3, consistent=False)
    orc = oracle.run(X, min_chain_reads=1)
    g = cg.cg_load_graph(ctx, X, min_chain_reads=1)
    try:
        part, _ = cg.cg_partition_contigs(g, 3, cg.WEIGHT_BASES)
        for p in range(3):
            check_part(g, orc, part, p)
    finally:
        g.close()

    keep = []

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        keep.append(t)                       # the pinned buffers outlive the graph
        return t.numpy()

    P = type("P", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(P, k, pinned(getattr(G, k)))
    orc = oracle.run(G)
    g = cg.cg_load_graph(ctx, P, flags=cg.HOST_READS)
    try:
        part, _ = cg.cg_partition_contigs(g, 4, cg.WEIGHT_READS)
        for p in range(4):
            check_part(g, orc, part, p)
    finally:
        g.close()


def test_part_errors(ctx):
    G = gen.generate("tiny-1Mb", threads=8)
    g = cg.cg_load_graph(ctx, G)
    try:
        nc, _ = cg.cg_emit_contigs(g)
        with pytest.raises(cg.CgError) as e:
            cg.cg_emit_part(g, np.zeros(nc - 1, np.int32), 0)
        assert e.value.status == cg.CG_EINVAL
        with pytest.raises(cg.CgError) as e:
            cg.cg_emit_part(g, None, 0)
        assert e.value.status == cg.CG_EINVAL
        with pytest.raises(ValueError):
            cg.cg_emit_part(g, np.zeros(nc, np.int64), 0)
        part = np.zeros(nc, np.int32)
        _, tot = cg.cg_emit_part(g, part, 0)
        with pytest.raises(cg.CgError) as e:    # output capacity below the part's bases
            cg.cg_emit_part(g, part, 0, np.empty(nc + 1, np.int64), np.empty(tot - 1, np.uint8))
        assert e.value.status == cg.CG_EINVAL
        off, bases = cg.contigs_host(g)        # still usable
        orc = oracle.run(G)
        assert np.array_equal(bases, orc.bases)
    finally:
        g.close()


def test_empty_graph(ctx):
    G = structured(3, [], [], lone=0)
    g = cg.cg_load_graph(ctx, G)
    try:
        nc, tot = cg.cg_emit_part(g, None, 0)
        assert (nc, tot) == (0, 0)
    finally:
        g.close()
