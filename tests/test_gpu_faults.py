"""Failure handling with host-side fault injection (no GPU fault, trap or
hang): each injected failure is reported with its status; CG_ECUDA,
CG_ETIMEOUT and CG_EKERNEL make the context refuse further work until it is
destroyed, CG_ENOMEM and CG_EGRAPH do not; a fresh context (or the same one,
for the recoverable ones) then gives bit-exact results. Server: admission
refusals and a stalled worker (a bounded wait gives up, the request still
completes)."""
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
