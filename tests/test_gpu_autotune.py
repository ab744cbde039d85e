"""The autotuner on the GPU: it times the grid on a real graph, caches the
choice, reuses it, and the chosen parameters give the same bytes."""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import autotune, cg

pytestmark = pytest.mark.gpu


def test_tune_cache_and_exact_output(tmp_path):
    from paper_2207_04350_gb300 import _build
    _build.build()
    G = gen.generate(gen.batched_graph(3), threads=8)
    orc = oracle.run(G, min_chain_reads=2)
    ctx = cg.cg_create(0)
    try:
        g = cg.cg_load_graph(ctx, G)
        cache = autotune.Cache(str(tmp_path / "t.json"))
        grid = autotune.GRID[:4]
        r1 = autotune.apply(ctx, g, (G.n, G.m, G.packed_bytes), cache=cache,
                            time_it=autotune.cuda_step_timer(ctx, g, reps=2), grid=grid)
        assert not r1["cached"] and r1["tuning"] in grid and r1["ms"] > 0
        assert cg.cg_get_tuning(ctx) == r1["tuning"]
        r2 = autotune.apply(ctx, g, (G.n, G.m, G.packed_bytes), cache=autotune.Cache(cache.path))
        assert r2["cached"] and r2["tuning"] == r1["tuning"]
        off, bases = cg.contigs_host(g)
        assert np.array_equal(off, orc.contig_off) and np.array_equal(bases, orc.bases)
        g.close()
    finally:
        ctx.close()
