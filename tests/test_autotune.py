"""Autotuner host logic on the CPU: selection, size classes and the JSON cache
(the timer is a stand-in; on a GPU it is CUDA events around the step)."""
import json

from paper_2207_04350_gb300 import autotune


def test_selects_the_fastest_and_breaks_ties_by_order():
    grid = [dict(ruler_log2=r, tile_bytes=32768, emit_blocks_per_sm=8, emit_block_threads=256) for r in (3, 4, 5)]
    times = {3: 1.2, 4: 1.0, 5: 1.0}
    best, ms = autotune.tune(lambda c: times[c["ruler_log2"]], grid)
    assert best["ruler_log2"] == 4 and ms == 1.0


def test_size_classes():
    a = autotune.size_class(6_200_000, 851_680, 23_278_360_544)
    assert a == autotune.size_class(5_000_000, 600_000, 20_000_000_000)
    assert a != autotune.size_class(333_333, 35_952, 1_000_000_000)
    assert autotune.size_class(0, 0, 0) == "n0-m0-p0"


def test_cache_round_trip_and_apply_uses_it(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "tune.json")
    calls = []

    class FakeCg:
        @staticmethod
        def cg_set_tuning(ctx, **t):
            calls.append(t)
    monkeypatch.setattr(autotune, "cg", FakeCg)
    c = autotune.Cache(path)
    timer_calls = []

    def timer(cand):
        timer_calls.append(cand)
        return 2.0 - 0.1 * cand["emit_blocks_per_sm"] - 0.01 * cand["ruler_log2"]
    r1 = autotune.apply(None, None, (1000, 854, 2_500_000), cache=c, device="GB300", time_it=timer)
    assert not r1["cached"] and len(timer_calls) == len(autotune.GRID)
    assert r1["tuning"] == {"ruler_log2": 5, "tile_bytes": 0, "emit_blocks_per_sm": 16, "emit_block_threads": 128}
    data = json.load(open(path))
    assert data["GB300"][r1["size_class"]]["tuning"] == r1["tuning"]
    # a new process reads the file; no timing happens for a known class
    c2 = autotune.Cache(path)
    r2 = autotune.apply(None, None, (1000, 854, 2_500_000), cache=c2, device="GB300",
                        time_it=lambda cand: 1 / 0)
    assert r2["cached"] and r2["tuning"] == r1["tuning"] and calls[-1] == r1["tuning"]
    # another device has its own entries
    r3 = autotune.apply(None, None, (1000, 854, 2_500_000), cache=c2, device="other", time_it=lambda cand: 1.0)
    assert not r3["cached"] and r3["tuning"] == autotune.GRID[0]


def test_unreadable_cache_is_rebuilt(tmp_path, monkeypatch):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    monkeypatch.setenv("CG_AUTOTUNE_CACHE", str(p))
    c = autotune.Cache()
    assert c.path == str(p) and c.data == {}
