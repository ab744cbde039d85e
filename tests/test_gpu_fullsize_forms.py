"""Parity of the batched and served forms at their full sizes, every graph
against the oracle:

- the 512-graph batch (genomes log-U[0.5, 12] Mb) as one union graph: every
  graph's contig offsets and bases, with the reads copied to the device and
  with them left in pinned host memory;
- the 200-graph served pool (genomes log-U[1, 200] Mb) through the server:
  every graph's contigs, alone and mixed into batches with other requests.
"""
import os

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


def _pinned_alloc(keep):
    import torch

    def alloc(shape, dt):
        t = torch.empty(shape, dtype=getattr(torch, dt.__name__), pin_memory=True)
        keep.append(t)
        return t.numpy()
    return alloc


def _oracle_all(graphs):
    """The oracle's contig offsets and bases of every graph. The oracle is
    single-threaded C called through ctypes (which releases the GIL), so the
    graphs run on a pool of threads."""
    import concurrent.futures as cf

    def one(G):
        w = oracle.run(G, min_chain_reads=2, validate=False)
        return w.n_contigs, w.total_bases, w.contig_off, w.bases
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, graphs))


def test_batched_512_full(ctx):
    """Every one of the 512 graphs of the batch, each graph's contig offsets and
    bases against the oracle run on that graph alone, with the reads copied to
    the device and with them left in pinned host memory."""
    keep = []
    alloc = _pinned_alloc(keep)
    graphs = [gen.generate(gen.batched_graph(j), keep_genome=False, alloc=alloc) for j in range(512)]
    want = _oracle_all(graphs)
    for flags in (0, cg.HOST_READS):
        g = cg.cg_load_batch(ctx, graphs, flags=flags, min_chain_reads=2)
        try:
            off, bases = cg.contigs_host(g)
            fc, fb = cg.cg_batch_ranges(g)
        finally:
            g.close()
        assert fc[0] == 0 and fb[0] == 0
        for j, (nc, tot, w_off, w_bases) in enumerate(want):
            assert fc[j + 1] - fc[j] == nc and fb[j + 1] - fb[j] == tot, j
            assert np.array_equal(off[fc[j]:fc[j + 1] + 1] - fb[j], w_off), j
            assert np.array_equal(bases[fb[j]:fb[j + 1]], w_bases), j
        assert fc[512] == len(off) - 1 and fb[512] == len(bases)


def test_served_pool_full(ctx):
    """Every one of the 200 graphs of the served pool through the server, against
    the oracle: once alone (one request per batch, one worker) and once mixed
    into batches (eight workers, as the bench serves, up to 64 requests per
    batch) by a seeded Poisson-order submission in which every graph appears at
    least once and some several times, so that each result is checked alone and
    in the mix."""
    import time
    keep = []
    alloc = _pinned_alloc(keep)
    P = 200
    pool = [gen.generate(gen.served_graph(j), keep_genome=False, alloc=alloc) for j in range(P)]
    want = _oracle_all(pool)

    def check(r, j):
        assert r["status"] == cg.CG_OK, j
        nc, tot, w_off, w_bases = want[j]
        assert r["n_contigs"] == nc and r["total_bases"] == tot, j
        assert np.array_equal(r["contig_off"], w_off), j
        assert np.array_equal(r["bases"], w_bases), j

    alone = cg.Server(0, hbm_budget_bytes=150 << 30, max_batch=1, workers=1)
    try:
        for j in range(P):
            rid = alone.submit(pool[j])
            r = alone.wait(rid)
            assert r["batch_size"] == 1
            check(r, j)
            alone.release(rid)
    finally:
        alone.stop()

    rng = np.random.default_rng(gen.SEED0 + 4)
    order = np.concatenate([rng.permutation(P), rng.integers(0, P, size=P)])
    gaps = rng.exponential(2e-4, size=len(order))
    mixed = cg.Server(0, hbm_budget_bytes=150 << 30, max_batch=64, workers=8)
    try:
        ids = []
        for j, gap in zip(order.tolist(), gaps.tolist()):
            time.sleep(gap)
            ids.append((mixed.submit(pool[j]), j))
        batch_sizes = []
        for rid, j in ids:
            r = mixed.wait(rid)
            check(r, j)
            batch_sizes.append(r["batch_size"])
            mixed.release(rid)
        assert max(batch_sizes) > 1, "no request was batched with another"
    finally:
        mixed.stop()
