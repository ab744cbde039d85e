"""Timing levels of a context (cg_set_timing): which stage times a step
records, and that timing never changes the output."""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg

pytestmark = pytest.mark.gpu


def test_timing_levels():
    import torch
    from paper_2207_04350_gb300 import _build
    _build.build()
    G = gen.generate("tiny-1Mb", threads=8)
    orc = oracle.run(G, min_chain_reads=2)
    ctx = cg.cg_create(0)
    try:
        src = type("D", (), {})()
        for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
            setattr(src, k, torch.from_numpy(np.ascontiguousarray(getattr(G, k))).cuda())
        g = cg.cg_load_graph(ctx, src, flags=cg.BORROW_DEVICE, min_chain_reads=2)
        n_contigs, total = cg.cg_emit_contigs(g)
        off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
        bases = torch.empty((total + 15) // 16 * 16, dtype=torch.uint8, device="cuda")

        def step():
            cg.cg_mask_branches(g, want_count=False)
            cg.cg_chains(g, want_counts=False)
            cg.cg_emit_contigs(g, off, bases, want_counts=False)
            return cg.cg_get_stats(ctx)["stage_ms"]

        for level, recorded in ((3, [False, False, False, True]), (1, [True] * 4), (2, [True] * 4),
                                (0, [False] * 4)):
            cg.cg_set_timing(ctx, level)
            for _ in range(2):                     # the first run of a level captures its graphs
                ms = step()
            cg.cg_sync(ctx)
            assert [t > 0 for t in ms] == recorded, (level, ms)
            if level == 2:
                names = [name for name, _ in cg.cg_kernel_times(ctx)]
                assert "k_mask" in names and "k_emit" in names
            assert np.array_equal(off.cpu().numpy(), orc.contig_off)
            assert np.array_equal(bases[:total].cpu().numpy(), orc.bases)
        g.close()
    finally:
        ctx.close()
