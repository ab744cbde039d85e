"""Failure handling with host-side fault injection (no GPU fault, trap or
hang): each injected failure is reported with its status; CG_ECUDA,
CG_ETIMEOUT and CG_EKERNEL make the context refuse further work until it is
destroyed, CG_ENOMEM and CG_EGRAPH do not; a fresh context (or the same one,
for the recoverable ones) then gives bit-exact results. Server: admission
refusals and a stalled worker (a bounded wait gives up, the request still
completes). One device wait really runs out: the look-back scan with its
first tile withheld returns by itself with CG_ETIMEOUT."""
import os

import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    import torch
    from paper_2207_04350_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    G = gen.generate("tiny-1Mb", threads=8)
    return G, oracle.run(G, min_chain_reads=2)


def contigs(ctx, G):
    g = cg.cg_load_graph(ctx, G)
    try:
        return cg.contigs_host(g)
    finally:
        g.close()


def exact(ctx, G, orc):
    off, bases = contigs(ctx, G)
    assert np.array_equal(off, orc.contig_off) and np.array_equal(bases, orc.bases)


def test_device_wait_runs_out(tiny):
    """A real device-side wait that runs out, not an injected status: the
    look-back scan with tile 0 withheld, so the later tiles wait on a
    descriptor that nothing publishes until their bounded wait gives up. The
    kernel returns by itself with CG_ETIMEOUT recorded; the context then
    refuses work, and a fresh context on the same GPU is bit-exact."""
    import time
    G, orc = tiny
    ctx = cg.cg_create(0)
    try:
        exact(ctx, G, orc)
        t0 = time.perf_counter()
        st = cg.cg_selftest_wait_timeout(ctx, 4)
        waited = time.perf_counter() - t0
        assert st == cg.CG_ETIMEOUT, cg.cg_status_str(st)
        assert waited < 30.0
        for call in (lambda: cg.cg_sync(ctx), lambda: contigs(ctx, G)):
            with pytest.raises(cg.CgError) as e:
                call()
            assert e.value.status == cg.CG_ETIMEOUT
    finally:
        ctx.close()
    ctx = cg.cg_create(0)
    try:
        exact(ctx, G, orc)
    finally:
        ctx.close()


@pytest.mark.parametrize("site,at,status,sticky", [
    ("alloc", 3, cg.CG_ENOMEM, False),
    ("bad_graph", 1, cg.CG_EGRAPH, False),
    ("h2d", 2, cg.CG_ECUDA, True),
    ("timeout", 2, cg.CG_ETIMEOUT, True),
    ("kernel", 1, cg.CG_EKERNEL, True),
])
def test_injected_failure(tiny, site, at, status, sticky):
    G, orc = tiny
    ctx = cg.cg_create(0)
    try:
        cg.cg_set_fault(ctx, f"{site}:{at}")
        with pytest.raises(cg.CgError) as e:
            contigs(ctx, G)
        assert e.value.status == status
        if sticky:
            with pytest.raises(cg.CgError) as e2:
                contigs(ctx, G)
            assert e2.value.status == status
        else:
            exact(ctx, G, orc)                   # the same context goes on
    finally:
        ctx.close()
    fresh = cg.cg_create(0)
    try:
        exact(fresh, G, orc)
    finally:
        fresh.close()


def test_plan_from_environment(tiny):
    G, orc = tiny
    os.environ["CG_FAULT"] = "bad_graph:2"
    try:
        ctx = cg.cg_create(0)
    finally:
        del os.environ["CG_FAULT"]
    try:
        exact(ctx, G, orc)                       # the first load passes
        with pytest.raises(cg.CgError) as e:
            contigs(ctx, G)
        assert e.value.status == cg.CG_EGRAPH
        exact(ctx, G, orc)
        cg.cg_set_fault(ctx, None)
    finally:
        ctx.close()


def server_with(plan, **kw):
    os.environ["CG_FAULT"] = plan
    try:
        return cg.Server(0, **kw)
    finally:
        del os.environ["CG_FAULT"]


def check_result(res, orc):
    assert res["status"] == cg.CG_OK
    assert np.array_equal(res["contig_off"], orc.contig_off) and np.array_equal(res["bases"], orc.bases)


def test_server_admission_refused(tiny):
    G, orc = tiny
    srv = server_with("admit:2", hbm_budget_bytes=8 << 30, max_batch=4, workers=2)
    try:
        a = srv.submit(G)
        with pytest.raises(cg.CgError) as e:
            srv.submit(G)
        assert e.value.status == cg.CG_EBUSY
        b = srv.submit(G)
        for rid in (a, b):
            check_result(srv.wait(rid), orc)
            srv.release(rid)
    finally:
        srv.stop()


def test_server_worker_stall(tiny):
    G, orc = tiny
    srv = server_with("queue_stall:1:600", hbm_budget_bytes=8 << 30, max_batch=4, workers=1)
    try:
        rid = srv.submit(G)
        with pytest.raises(cg.CgError) as e:
            srv.wait(rid, timeout_ms=50)          # the worker is stalled: the bounded wait gives up
        assert e.value.status == cg.CG_ETIMEOUT
        check_result(srv.wait(rid), orc)         # and the request still completes
        srv.release(rid)
    finally:
        srv.stop()


def test_server_replaces_a_refusing_context(tiny):
    """A batch whose device wait reports a timeout leaves its context refusing
    work; the worker replaces that context, so the failed batch's request
    reports CG_ETIMEOUT and every later request is bit-exact."""
    G, orc = tiny
    srv = server_with("batch_timeout:1", hbm_budget_bytes=8 << 30, max_batch=4, workers=1)
    try:
        rid = srv.submit(G)
        res = srv.wait(rid)
        assert res["status"] == cg.CG_ETIMEOUT
        srv.release(rid)
        for _ in range(3):
            rid = srv.submit(G)
            check_result(srv.wait(rid), orc)
            srv.release(rid)
        assert srv.stats()["contexts_replaced"] == 1
    finally:
        srv.stop()


def test_server_malformed_request_fails_alone(tiny):
    """One malformed graph batched with valid ones: the union fails its input
    checks, the batch is run again one request at a time, and only the
    malformed request reports CG_EGRAPH; the others are bit-exact."""
    G, orc = tiny
    B = type("B", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(B, k, np.array(getattr(G, k), copy=True))
    B.code[0] ^= 1                                # the entry no longer matches its mirror
    assert not oracle.validate(B)[0]
    # the first batch stalls, so the requests submitted meanwhile form one batch
    srv = server_with("queue_stall:1:500", hbm_budget_bytes=8 << 30, max_batch=16, workers=1)
    try:
        first = srv.submit(G)
        ids = [(srv.submit(B if i == 2 else G), i == 2) for i in range(5)]
        check_result(srv.wait(first), orc)
        srv.release(first)
        for rid, bad in ids:
            res = srv.wait(rid)
            if bad:
                assert res["status"] == cg.CG_EGRAPH
            else:
                check_result(res, orc)
            srv.release(rid)
        assert srv.stats()["batches"] == 2       # the five shared one batch
    finally:
        srv.stop()
