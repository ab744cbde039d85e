"""Launch-parameter autotuning for the contig path, with a JSON cache.

The parameters (cg_tuning: the sublist sampling 2^-ruler_log2, the emission
tile size, resident emission blocks per SM and the emission CTA size) never
change an output byte; they only move time between the chain stage and the
spelling. This module times a
small grid of them on a loaded graph (the whole step: cg_mask_branches ->
cg_chains -> cg_emit_contigs into device buffers, waited for), keeps the
fastest by median, and caches the choice per size class of the input
(powers of two of reads, overlap entries and packed bytes) and device name.
The cache file is CG_AUTOTUNE_CACHE, else ~/.cache/paper_2207_04350_gb300/
autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

from . import cg

# (resident blocks per SM, threads per block) of the spelling kernels: half
# occupancy, and full occupancy with CTAs of 256, 128 and 512 threads (the
# blocks per SM are capped at what fits)
LAUNCH = ((4, 256), (8, 256), (16, 128), (2, 512))
# spelling tile: 0 lets each launch choose from its output size
GRID = [dict(ruler_log2=r, tile_bytes=t, emit_blocks_per_sm=b, emit_block_threads=bt)
        for r in (3, 4, 5) for t in (0, 16384, 32768, 65536) for b, bt in LAUNCH]


def size_class(n_reads: int, n_entries: int, packed_bytes: int) -> str:
    """Inputs within a factor of two of each other share a tuning."""
    lg = (lambda x: int(math.ceil(math.log2(x))) if x > 1 else 0)
    return f"n{lg(n_reads)}-m{lg(n_entries)}-p{lg(packed_bytes)}"


def default_path() -> str:
    return os.environ.get("CG_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2207_04350_gb300", "autotune.json")


class Cache:
    """{device name: {size class: {"tuning": {...}, "ms": median ms, "candidates": n}}} in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path or default_path()
        self._lock = threading.Lock()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}             # an unreadable cache is rebuilt

    def get(self, device: str, key: str):
        return self.data.get(device, {}).get(key)

    def put(self, device: str, key: str, entry: dict):
        with self._lock:
            self.data.setdefault(device, {})[key] = entry
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            tmp = self.path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def device_name(index: int = 0) -> str:
    import torch
    return torch.cuda.get_device_name(index)


def cuda_step_timer(ctx, g, reps: int = 5):
    """A timer for `tune`: runs the step once to warm up, then `reps` times, each
    waited for (cg_sync), and returns the median wall time (ms). The waits cost
    the same for every candidate, so the order of candidates is the order of
    their GPU times."""
    import time
    import torch
    n_contigs, total = cg.cg_emit_contigs(g)
    off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
    bases = torch.empty(max(16, (total + 15) // 16 * 16), dtype=torch.uint8, device="cuda")

    def step():
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        cg.cg_emit_contigs(g, off, bases, want_counts=False)
        cg.cg_sync(ctx)

    def time_it(tuning: dict) -> float:
        cg.cg_set_tuning(ctx, **tuning)
        step()
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            step()
            times.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(times)
    return time_it


def tune(time_it, grid=None) -> tuple[dict, float]:
    """The candidate of `grid` with the smallest time_it(candidate), and that time;
    ties go to the earlier candidate."""
    best, best_ms = None, float("inf")
    for cand in grid or GRID:
        ms = float(time_it(dict(cand)))
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    return best, best_ms


def apply(ctx, g, graph_sizes: tuple[int, int, int], cache: Cache | None = None, device: str | None = None,
          time_it=None, grid=None) -> dict:
    """Sets the context's tuning for graph g from the cache, tuning and caching it
    first when its size class is new. graph_sizes = (reads, entries, packed bytes).
    Returns {"tuning", "ms", "cached"}."""
    cache = cache or Cache()
    device = device or device_name()
    key = size_class(*graph_sizes)
    hit = cache.get(device, key)
    if hit is not None:
        cg.cg_set_tuning(ctx, **hit["tuning"])
        return {"tuning": hit["tuning"], "ms": hit["ms"], "cached": True, "size_class": key}
    time_it = time_it or cuda_step_timer(ctx, g)
    best, ms = tune(time_it, grid)
    cache.put(device, key, {"tuning": best, "ms": ms, "candidates": len(grid or GRID)})
    cg.cg_set_tuning(ctx, **best)
    return {"tuning": best, "ms": ms, "cached": False, "size_class": key}
