"""GreedyPartitioning (Sec. 4.3) on the GPU against the oracle's LPT rule.

The contig weights (reads per contig, or spelled bases) come from the oracle's
own contig generation; the GPU sorts and assigns on its side from its own
contigs. Part of every contig and weight sum of every part: bit-exact. Cases
cover many equal weights (ties in the sort and in the least-loaded choice),
more than one sort tile (2048 contigs) with a ragged tail, part counts below,
at and above one warp (32) up to the limit, and more parts than contigs.
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


def oracle_weights(orc, weight):
    if weight == cg.WEIGHT_BASES:
        return np.diff(orc.contig_off).astype(np.int64)
    ids, counts = np.unique(orc.chain_id[orc.chain_id >= 0], return_counts=True)
    assert len(ids) == orc.n_contigs       # contigs are listed by their smallest read
    return counts.astype(np.int64)


def check(ctx, G, parts, mcr=2, device=False):
    orc = oracle.run(G, min_chain_reads=mcr)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    try:
        for weight in (cg.WEIGHT_READS, cg.WEIGHT_BASES):
            w = oracle_weights(orc, weight)
            for P in parts:
                want_part, want_sum = oracle.lpt(w, P)
                if device:
                    import torch
                    part_t = torch.full((max(orc.n_contigs, 1),), -7, dtype=torch.int32, device="cuda")
                    sum_t = torch.empty(P, dtype=torch.int64, device="cuda")
                    nc = cg.cg_partition_contigs(g, P, weight, part_t, sum_t)
                    got_part, got_sum = part_t.cpu().numpy()[:nc], sum_t.cpu().numpy()
                else:
                    got_part, got_sum = cg.cg_partition_contigs(g, P, weight)
                assert len(got_part) == orc.n_contigs
                assert np.array_equal(got_part, want_part), (weight, P)
                assert np.array_equal(got_sum, want_sum), (weight, P)
    finally:
        g.close()


def test_tiny_workload(ctx):
    G = gen.generate("tiny-1Mb", threads=4)
    check(ctx, G, [1, 2, 3, 8, 31, 32, 33, 64, 65, 72, 128, 129, 200, 256, 300, 512, 513, 1024])


def test_wide_keys(ctx):
    """Weight sums of more than 2^22 bases with 1024 parts: keys beyond 32 bits."""
    G = gen.generate(dict(gen.WORKLOADS["tiny-1Mb"](), genome_len=8_000_000), threads=8)
    orc = oracle.run(G)
    assert orc.total_bases << 10 > 2**32
    check(ctx, G, [8, 72, 300, 1024])


def test_ties_and_sort_tiles(ctx):
    rng = np.random.default_rng(11)
    # 5000 chains of a few sizes: long runs of equal weights, 3 sort tiles
    sizes = list(rng.choice([2, 3, 4, 7], size=5000))
    G = structured(4, sizes, lone=300)
    check(ctx, G, [1, 5, 32, 64, 1000, 1024])
    check(ctx, G, [7, 33], device=True)


def test_more_parts_than_contigs(ctx):
    G = structured(8, [2, 5, 3], lone=2)
    check(ctx, G, [1, 2, 3, 4, 40, 1024], mcr=1)
    check(ctx, G, [50], device=True)


def test_no_contigs(ctx):
    G = structured(9, [], lone=5)
    orc = oracle.run(G)
    assert orc.n_contigs == 0
    g = cg.cg_load_graph(ctx, G)
    try:
        part, psum = cg.cg_partition_contigs(g, 4)
        assert len(part) == 0 and np.array_equal(psum, np.zeros(4, np.int64))
    finally:
        g.close()


def test_bad_arguments(ctx):
    G = structured(3, [3, 4])
    g = cg.cg_load_graph(ctx, G)
    try:
        for P in (0, -1, cg.MAX_PARTS + 1):
            with pytest.raises(cg.CgError):
                cg.cg_partition_contigs(g, P)
        with pytest.raises(cg.CgError):
            cg.cg_partition_contigs(g, 2, weight=5)
        small = np.empty(1, np.int32)
        with pytest.raises(cg.CgError):
            cg.cg_partition_contigs(g, 2, cg.WEIGHT_READS, small, np.empty(2, np.int64))
        part, psum = cg.cg_partition_contigs(g, 2)    # the context is still usable
        assert len(part) == 2
    finally:
        g.close()


def test_many_contigs_few_parts(ctx):
    """9,000 and 17,000 contigs of a few read counts (long runs of equal
    weights, several sort tiles) into 2 to 32 parts."""
    rng = np.random.default_rng(12)
    G = structured(6, list(rng.choice([2, 3, 5, 8, 13, 40], size=9000)), lone=10)
    check(ctx, G, [2, 7, 8, 9, 16, 17, 31, 32])
    G = structured(7, list(rng.choice([2, 3, 4], size=17000)), lone=10)
    check(ctx, G, [8, 16, 32])


def test_one_contig_of_80mb(ctx):
    """A contig of about 80 Mb with 3 and 32 parts: part sums beyond 32 bits
    once shifted above the part index, so the assignment takes wide keys."""
    G = structured(13, [4000, 30, 20, 10, 5, 5, 3, 2, 2, 2], min_len=40000, max_len=40000)
    orc = oracle.run(G)
    assert (2 * int(np.diff(orc.contig_off).max()) + 1) << 5 > 2**32
    check(ctx, G, [3, 32])


@pytest.mark.slow
def test_genome_100mb(ctx):
    G = gen.generate("genome-100Mb", threads=16)
    check(ctx, G, [8, 72, 1024])


def test_kernel_marks(ctx):
    """Per-kernel timing marks with graphs off and on, over a run and a partition."""
    G = structured(5, [4, 6, 9, 2], lone=3)
    for graphs in (False, True):
        cg.cg_set_graphs(ctx, graphs)
        cg.cg_set_timing(ctx, 2)
        try:
            g = cg.cg_load_graph(ctx, G)
            try:
                cg.contigs_host(g)
                names = [n for n, _ in cg.cg_kernel_times(ctx)]
                assert "k_mask" in names and "k_emit" in names
                cg.cg_partition_contigs(g, 3)
                t = cg.cg_kernel_times(ctx)
                assert [n for n, _ in t][-1] == "k_lpt_assign" and all(ms >= 0 for _, ms in t)
            finally:
                g.close()
        finally:
            cg.cg_set_timing(ctx, 0)
            cg.cg_set_graphs(ctx, True)
