"""TransitiveReduction (Alg. 1, Sec. 2) on the GPU (cg_transitive_reduction)
against the oracle, entry for entry (row offsets, columns, codes, suffixes),
and against the interval property at the 100 Mb size: the reduction of every
exact overlap among reads of one genome is the consecutive-overlap graph.
The reduced graph then goes through the contig path on the device."""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg
from tests import _pins
from tests._gpu import assert_parity, run_gpu

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


def same_csr(a, b):
    for k in ("row_ptr", "col", "code", "suf"):
        x, y = np.asarray(getattr(a, k)), np.asarray(getattr(b, k))
        if x.shape != y.shape or not np.array_equal(x.astype(np.int64), y.astype(np.int64)):
            return False
    return True


def test_hand_cases(ctx):
    rows = [((1, 1, 1), (10, 15, 25, 30, 20, 50), 0), ((1, 1, 0), (10, 15, 25, 30, 20, 50), 0),
            ((1, 0, 1), (10, 15, 25, 30, 20, 50), 0), ((1, 1, 3), (10, 15, 25, 30, 20, 50), 0),
            ((1, 1, 1), (10, 15, 26, 30, 20, 51), 0), ((1, 1, 1), (10, 15, 26, 30, 20, 51), 1),
            ((1, 1, 1), (10, 15, 26, 30, 20, 50), 0), ((3, 2, 3), (10, 15, 25, 30, 20, 50), 0)]
    for codes, sufs, fuzz in rows:
        G = _pins._tr_triangle(*codes, *sufs)
        assert same_csr(cg.cg_transitive_reduction(ctx, G, fuzz), oracle.transitive_reduction(G, fuzz))


@pytest.mark.parametrize("fuzz", [0, 40])
def test_generated_with_repeats(ctx, fuzz):
    cfgs = [dict(gen.WORKLOADS["tiny-1Mb"](), full_overlaps=1),
            dict(gen._cfg(91, 600_000, [(0.08, 2000, 6000, 3, 10, 0.0)], 15, 1, 7000, 3000, 2500), full_overlaps=1),
            dict(gen._cfg(92, 800_000, [(0.1, 3000, 8000, 2, 12, 0.05)], 20, 0, 5000, 15000, 2500),
                 full_overlaps=1, rep_div_accept=0.1)]
    for d in cfgs:
        R = gen.generate(d, threads=8, off_align=1)
        S = cg.cg_transitive_reduction(ctx, R, fuzz)
        assert S.m < R.m
        assert same_csr(S, oracle.transitive_reduction(R, fuzz))


def test_noisy_suffixes(ctx):
    R = gen.generate(dict(gen.WORKLOADS["tiny-1Mb"](), full_overlaps=1), threads=8)
    rng = np.random.default_rng(3)
    N = type("N", (), {})()
    for k in ("row_ptr", "col", "code", "len", "off", "packed"):
        setattr(N, k, getattr(R, k))
    lv = np.asarray(R.len)[np.asarray(R.col)]
    N.suf = np.clip(np.asarray(R.suf) + rng.integers(-3, 4, size=R.m), 1, lv - 1).astype(np.int32)
    for fuzz in (0, 2, 6):
        assert same_csr(cg.cg_transitive_reduction(ctx, N, fuzz), oracle.transitive_reduction(N, fuzz))


def test_interval_property_100mb(ctx):
    d = dict(gen.WORKLOADS["genome-100Mb"](), k_rep=0)
    full = gen.generate(dict(d, full_overlaps=1), threads=16)
    red = gen.generate(d, threads=16)
    assert full.m > 3 * red.m
    S = cg.cg_transitive_reduction(ctx, full)
    assert same_csr(S, red)


def test_on_device_to_contigs(ctx):
    import torch
    R = gen.generate(dict(gen.WORKLOADS["tiny-1Mb"](), full_overlaps=1), threads=8)
    dev = type("D", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(dev, k, torch.from_numpy(np.ascontiguousarray(getattr(R, k))).cuda())
    S = cg.cg_transitive_reduction(ctx, dev, device=True)
    S.len, S.off, S.packed = dev.len, dev.off, dev.packed
    host = type("H", (), {})()
    for k in ("row_ptr", "col", "code", "suf"):
        setattr(host, k, getattr(S, k).cpu().numpy())
    host.len, host.off, host.packed = R.len, R.off, R.packed
    assert same_csr(host, oracle.transitive_reduction(R))
    orc = oracle.run(host, min_chain_reads=2)
    g = cg.cg_load_graph(ctx, S, flags=cg.BORROW_DEVICE, min_chain_reads=2)
    try:
        off, bases = cg.contigs_host(g)
    finally:
        g.close()
    assert np.array_equal(off, orc.contig_off) and np.array_equal(bases, orc.bases)


def test_invalid_and_capacity(ctx):
    G = _pins._tr_triangle(1, 1, 1, 10, 15, 25, 30, 20, 50)
    bad = []
    for k, i, v in (("col", 0, 2), ("col", 0, 9), ("code", 0, 4), ("suf", 0, 0)):
        H = type("H", (), {})()
        for f in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
            setattr(H, f, np.array(getattr(G, f), copy=True))
        getattr(H, f if False else k)[i] = v
        bad.append(H)
    for H in bad:
        with pytest.raises(cg.CgError) as e:
            cg.cg_transitive_reduction(ctx, H)
        assert e.value.status == cg.CG_EGRAPH
    import ctypes
    from paper_2207_04350_gb300.cg import _desc, lib
    d = _desc(G, 2)
    rp = np.empty(4, np.int64)
    small = np.empty(1, np.int32), np.empty(1, np.uint8), np.empty(1, np.int32)
    cnt = ctypes.c_int64(-1)
    st = lib().cg_transitive_reduction(ctx.ptr, ctypes.byref(d), 0, rp.ctypes.data, small[0].ctypes.data,
                                       small[1].ctypes.data, small[2].ctypes.data, 1, cg.MEM_HOST, ctypes.byref(cnt))
    assert st == cg.CG_EINVAL and cnt.value == 4
    S = cg.cg_transitive_reduction(ctx, G)         # still usable
    assert S.m == 4
