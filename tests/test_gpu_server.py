"""Served form: continuous batching gives every request exactly the contigs
it gets alone (the oracle), whatever it was batched with, under a tight
admission budget too."""
import time

import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    from paper_2207_04350_gb300 import _build
    _build.build()
    graphs = [gen.generate(gen.batched_graph(j), threads=8) for j in range(12)]
    graphs.append(gen.generate("tiny-1Mb", threads=8))
    want = [oracle.run(G, min_chain_reads=2) for G in graphs]
    return graphs, want


def _check(res, want):
    assert res["status"] == cg.CG_OK
    assert res["n_contigs"] == want.n_contigs
    assert np.array_equal(res["contig_off"], want.contig_off)
    assert np.array_equal(res["bases"], want.bases)


def test_each_result_is_the_same_alone_and_in_the_mix(pool):
    graphs, want = pool
    # alone: one request at a time
    srv = cg.Server(0, hbm_budget_bytes=64 << 30, max_batch=1, workers=1)
    try:
        for j in range(0, len(graphs), 4):
            rid = srv.submit(graphs[j])
            _check(srv.wait(rid), want[j])
            srv.release(rid)
    finally:
        srv.stop()
    # in the mix: 60 requests over the pool submitted at once
    srv = cg.Server(0, hbm_budget_bytes=64 << 30, max_batch=16, workers=2)
    try:
        ids = [(srv.submit(graphs[i % len(graphs)]), i % len(graphs)) for i in range(60)]
        sizes = []
        for rid, j in ids:
            res = srv.wait(rid)
            _check(res, want[j])
            sizes.append(res["batch_size"])
            srv.release(rid)
        st = srv.stats()
        assert st["requests"] == 60 and st["in_flight_bytes"] == 0
        assert max(sizes) > 1 and st["batches"] < 60          # requests really shared batches
    finally:
        srv.stop()


def test_tight_budget_queues_but_stays_exact(pool):
    graphs, want = pool
    est = max(2 * G.packed.nbytes + 400 * G.n + 16 * G.m + (1 << 20) for G in graphs)
    srv = cg.Server(0, hbm_budget_bytes=int(2.5 * est), max_batch=8, workers=2)
    try:
        ids = [(srv.submit(graphs[i % len(graphs)]), i % len(graphs)) for i in range(30)]
        for rid, j in ids:
            _check(srv.wait(rid), want[j])
            srv.release(rid)
        assert srv.stats()["in_flight_bytes"] == 0
        with pytest.raises(cg.CgError) as e:
            big = cg.Server(0, hbm_budget_bytes=1 << 20, max_batch=1, workers=1)
            try:
                big.submit(graphs[0])
            finally:
                big.stop()
        assert e.value.status == cg.CG_EBUSY
    finally:
        srv.stop()


def test_poll_and_timestamps(pool):
    graphs, want = pool
    srv = cg.Server(0, hbm_budget_bytes=16 << 30, max_batch=4, workers=2)
    try:
        rid = srv.submit(graphs[-1])
        t_end = time.time() + 60
        while not srv.poll(rid) and time.time() < t_end:
            time.sleep(0.001)
        res = srv.wait(rid, timeout_ms=60_000)
        _check(res, want[-1])
        assert res["t_submit_ns"] <= res["t_start_ns"] <= res["t_done_ns"]
        srv.release(rid)
    finally:
        srv.stop()
