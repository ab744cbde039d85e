#!/usr/bin/env python
"""Contig-generation benchmark on GB300: contig Gbases/s of the plain path.

One step = one pass of the whole path over one string graph: branch masking,
successor table, list ranking, contig sizes and order, compaction by chain,
piece offsets and spelling (cg_mask_branches -> cg_chains -> cg_emit_contigs),
with the graph and the reads resident in HBM. The default workload is the
3.1 Gb genome-shaped graph (6.2M reads, 23 GB of 2-bit packed reads).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line (rank 0). With --gpus N > 1 under torchrun every rank
runs an independent replica of the workload (the path needs no cross-GPU
exchange) and the time is the maximum over ranks. --impl reference times the
CPU oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contig Gbases/s & ms per graph (plain vs batched) vs HBM roofline; p50/p99 latency"
UNIT = "Gbases/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# DRAM bytes (read + write) per contig base of k_emit from one ncu capture
# (--set full, the 3.1 Gb recipe on a 450 Mb genome: 552.2 MB for 481,446,585
# bases), valid only for the emission source it was taken on.
EMIT_TRAFFIC = {"bytes_per_base": (128.766464e6 + 421.409280e6) / 481446585, "source_sha256_16": "81bd7d9611aecfe5"}


def _reduce(x: float, world: int, op: str) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the slowest replica's time); x on one rank."""
    return _reduce(x, world, "max")


def sum_over_ranks(x: float, world: int) -> float:
    """The sum of x over all ranks (units every replica processed); x on one rank."""
    return _reduce(x, world, "sum")


def rank_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(units_per_rank: float, seconds_per_rank: float, world: int) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return sum_over_ranks(units_per_rank, world) / max_over_ranks(seconds_per_rank, world)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", default="genome-3.1Gb",
                   help="tiny-1Mb | genome-100Mb | genome-3.1Gb | batched-512 | served-2000")
    p.add_argument("--batch-graphs", type=int, default=512, help="graphs of the batched workload")
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-pool", type=int, default=200, help="pre-generated graphs the requests draw from")
    p.add_argument("--serve-budget-gb", type=float, default=150.0)
    p.add_argument("--serve-max-batch", type=int, default=64)
    p.add_argument("--serve-workers", type=int, default=8, help="worker threads (contexts, streams) of the server")
    p.add_argument("--serve-load", type=float, default=0.8, help="offered load / plain one-at-a-time throughput")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=5.0, help="CPU budget of the scaled oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--shard", default="", choices=["", "tiles", "lpt"],
                   help="split one graph over the ranks (strong scaling) instead of one replica per rank")
    p.add_argument("--no-forms", action="store_true",
                   help="main workload only: skip the compact records of the other four workloads")
    p.add_argument("--no-transitive", action="store_true", help="skip the transitive-reduction measurement")
    p.add_argument("--pg-timeout", type=int, default=300, help="process-group timeout (s) for N > 1")
    p.add_argument("--autotune", action="store_true",
                   help="tune the launch parameters for this size class first (cached as JSON)")
    p.add_argument("--min-chain-reads", type=int, default=2)
    p.add_argument("--threads", type=int, default=0, help="generator threads (0 = all cores)")
    p.add_argument("--scale-genome", type=int, default=0,
                   help="profiling only: the workload's recipe on a genome of this many bases")
    p.add_argument("--ruler-log2", type=int, default=0)
    p.add_argument("--tile-bytes", type=int, default=0)
    p.add_argument("--emit-blocks-per-sm", type=int, default=0)
    p.add_argument("--emit-block-threads", type=int, default=0, help="spelling CTA size: 128, 256 or 512")
    p.add_argument("--partition-parts", type=int, nargs="*", default=[8, 18, 72, 128],
                   help="part counts for the GreedyPartitioning measurement (none: skip)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"])}, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, reasons) taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if t0 <= t <= t1 and len(r) >= 9]
        window = "timed region"
        if not rows:
            rows = [r for _, r in self.rows if len(r) >= 9]
            window = "whole run (timed region shorter than the 100 ms sampling period)"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window}


# -------------------------------------------------------------- workload
def workload_cfg(name):
    import gen
    if name not in gen.WORKLOADS:
        raise SystemExit(f"unknown workload {name}; one of {sorted(gen.WORKLOADS)}")
    return gen.WORKLOADS[name]()


def generate_pinned(cfg, threads):
    import torch

    import gen
    keep = []

    def alloc(shape, dt):
        t = torch.empty(shape, dtype=getattr(torch, dt.__name__ if hasattr(dt, "__name__") else str(dt)),
                        pin_memory=True)
        keep.append(t)
        return t.numpy()
    G = gen.generate(cfg, threads=threads or None, alloc=alloc, keep_genome=False)
    G._pinned = keep
    return G


def bmin_bytes(G, W, total, C):
    """Least bytes any implementation moves: row_ptr, every CSR entry once,
    len+off of the spelled reads, the 2-bit bases spelled, the ASCII output
    and the contig offsets."""
    rp = G.row_ptr.dtype.itemsize
    return (G.n + 1) * rp + 9 * G.m + 12 * W + (total + 3) // 4 + total + 8 * (C + 1)


# --------------------------------------------------------------- ours
def run_batched(args, rank, world, local_rank):
    """512 graphs (log-uniform 0.5-12 Mb genomes): one union graph run as one
    pass of each stage, against the same graphs run one by one (plain)."""
    import torch

    import gen
    from paper_2207_04350_gb300 import cg

    torch.cuda.set_device(local_rank)
    pk, pk_kind = peaks()
    k = args.batch_graphs
    t_gen = time.time()
    graphs = [generate_pinned(gen.batched_graph(j), args.threads) for j in range(k)]
    t_gen = time.time() - t_gen
    stream = torch.cuda.Stream()
    ctx = cg.cg_create(local_rank, stream=stream)
    cg.cg_set_tuning(ctx, args.ruler_log2, args.tile_bytes, args.emit_blocks_per_sm, args.emit_block_threads)
    mcr = args.min_chain_reads
    # plain: every graph loaded on its own (untimed), outputs sized by a size query
    plain = []
    for G in graphs:
        g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
        nc, tot = cg.cg_emit_contigs(g)
        plain.append((g, torch.empty(nc + 1, dtype=torch.int64, device="cuda"),
                      torch.empty(max(16, (tot + 15) // 16 * 16), dtype=torch.uint8, device="cuda"), tot))
    union = cg.cg_load_batch(ctx, graphs, min_chain_reads=mcr)
    n_contigs, total = cg.cg_emit_contigs(union)
    assert total == sum(p[3] for p in plain)
    u_off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
    u_bases = torch.empty(max(16, (total + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def run_plain():
        for g, off, bases, _ in plain:
            cg.cg_mask_branches(g, want_count=False)
            cg.cg_chains(g, want_counts=False)
            cg.cg_emit_contigs(g, off, bases, want_counts=False)

    def run_union():
        cg.cg_mask_branches(union, want_count=False)
        cg.cg_chains(union, want_counts=False)
        cg.cg_emit_contigs(union, u_off, u_bases, want_counts=False)

    cg.cg_set_timing(ctx, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps, warmup, emit_times=None):
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            fn()
        cg.cg_sync(ctx)
        out = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(2)
            ev0.record(stream)
            fn()
            ev1.record(stream)
            ev1.synchronize()
            st = cg.cg_get_stats(ctx)
            out.append(ev0.elapsed_time(ev1))
            if emit_times is not None:
                emit_times.append(st["stage_ms"][3])
        cg.cg_sync(ctx)
        return statistics.mean(out)

    plain_steps = max(1, min(args.steps, 5))
    cg.cg_set_timing(ctx, 0)            # no events inside the baseline's steps
    ms_plain = timed(run_plain, plain_steps, 1)
    cg.cg_set_timing(ctx, 3)            # timed steps: events around the spelling stage only
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    launches0 = cg.cg_get_stats(ctx)["kernels_launched"]
    emit_ms = []
    rank_barrier(world)
    t0 = time.time()
    ms_rank = timed(run_union, args.steps, args.warmup, emit_ms)
    rank_barrier(world)
    t1 = time.time()
    value = job_rate(total, ms_rank * 1e-3, world) / 1e9
    ms = max_over_ranks(ms_rank, world)
    launches = cg.cg_get_stats(ctx)["kernels_launched"] - launches0
    time.sleep(0.2)
    clocks.stop()
    kern = {}
    cg.cg_set_timing(ctx, 2)
    for _ in range(3):
        run_union()
        for name, kms in cg.cg_kernel_times(ctx):
            kern.setdefault(name, []).append(kms)
    cg.cg_set_timing(ctx, 1)
    ms_emit = statistics.mean(emit_ms)
    # end to end: the batch from pinned host buffers, outputs back to pinned host buffers
    e2e = None
    e2e_copy = None
    if not args.no_e2e and args.e2e_steps > 0:
        h_bases = torch.empty(max(total, 1), dtype=torch.uint8, pin_memory=True).numpy()
        h_off = torch.empty(n_contigs + 1, dtype=torch.int64, pin_memory=True).numpy()
        names = ("row_ptr", "col", "code", "suf", "len", "off", "packed")
        copied = sum(getattr(G, k2).nbytes for G in graphs for k2 in names if k2 != "packed")
        d2h = total + 8 * (n_contigs + 1) + 16 * (k + 1)

        def e2e_run(flags):
            times = []
            for i in range(args.e2e_steps + 1):
                torch.cuda.synchronize()
                a = time.perf_counter()
                gu = cg.cg_load_batch(ctx, graphs, flags=flags, min_chain_reads=mcr)
                cg.cg_mask_branches(gu, want_count=False)
                cg.cg_chains(gu, want_counts=False)
                cg.cg_emit_contigs(gu, h_off, h_bases)
                fc, fb = cg.cg_batch_ranges(gu)
                gu.close()
                b = time.perf_counter()
                if i > 0:
                    times.append(b - a)
            return statistics.mean(times), len(times)
        te, ne = e2e_run(cg.HOST_READS)
        e2e = {"value": job_rate(total, te, world) / 1e9, "unit": UNIT, "h2d_bytes_per_step": copied + (total + 3) // 4,
               "d2h_bytes_per_step": d2h, "ms_per_step": te * 1e3, "graphs_per_s": k / te, "steps": ne,
               "h2d_note": "graph arrays copied + the 2-bit bases of the spelled pieces, gathered from each graph's "
                           "pinned reads over the host link",
               "path": "cg_load_batch(host, validated, CG_HOST_READS) -> mask -> chains -> cg_emit_contigs(pinned "
                       "host outputs) -> cg_batch_ranges"}
        tc, nc2 = e2e_run(0)
        e2e_copy = {"value": job_rate(total, tc, world) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": sum(getattr(G, k2).nbytes for G in graphs for k2 in names),
                    "d2h_bytes_per_step": d2h, "ms_per_step": tc * 1e3, "graphs_per_s": k / tc, "steps": nc2,
                    "path": "cg_load_batch(host, validated: every input copied) -> mask -> chains -> "
                            "cg_emit_contigs(pinned host outputs) -> cg_batch_ranges"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # every graph's slice of the union's last output against the oracle on that graph
        h_uoff, h_ubases = u_off.cpu().numpy(), u_bases[:total].cpu().numpy()
        fc, fb = cg.cg_batch_ranges(union)
        cpu = oracle_leg(graphs, lambda j: (h_uoff[fc[j]:fc[j + 1] + 1] - fb[j], h_ubases[fb[j]:fb[j + 1]]), mcr,
                         what=f"batched-{k}")
        del h_uoff, h_ubases
    emit_bytes = total + (total + 3) // 4
    ach = emit_bytes / (ms_emit * 1e-3) / 1e9
    n_reads = sum(G.n for G in graphs)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_per_graph": ms / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (the seeded generator gen/: genome, repeats, reads and overlaps of the stated recipe)",
        "config": {
            "workload": f"batched-{k} (graphs log-U[0.5,12] Mb genome, 2% repeats, 30x, LN(10 kb, 5 kb))",
            "graphs": k, "n_reads": n_reads, "contig_bases": total, "n_contigs": n_contigs,
            "tuning": cg.cg_get_tuning(ctx), "min_chain_reads": mcr,
            "e2e_copy_all_inputs": e2e_copy, "graphs_per_s_batched": k / (ms * 1e-3), "graphs_per_s_plain": k / (ms_plain * 1e-3),
            "ms_per_graph_batched": ms / k, "ms_per_graph_plain": ms_plain / k,
            "batched_over_plain": ms_plain / ms, "plain_steps": plain_steps,
            "plain": "the same graphs loaded one by one, mask/chains/emit per graph, all launches back to back",
            "l2": "flushed between steps (512 MiB write, outside the timed events)",
            "events": "timed steps record CUDA events around the spelling stage only (its live launch time); "
                      "the stage and kernel breakdowns come from separate untimed steps",
            "kernel_ms_mean": {kk: statistics.mean(v) for kk, v in kern.items()},
            "generate_s": round(t_gen, 1), "wall_s_timed": t1 - t0,
        },
        "roofline": {"kernel": "k_emit (contig spelling)", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": None,
                     "algorithmic_bytes_per_launch": emit_bytes, "bytes_per_unit": 1.25,
                     "units_per_launch": total, "ms_per_launch": ms_emit, "peak_kind": pk_kind + " (hbm_gbs, copy)"},
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks.summary(t0, t1), "gpu_launches": launches,
    }
    for g, _, _, _ in plain:
        g.close()
    union.close()
    ctx.close()
    return line


def run_served(args, rank, world, local_rank):
    """A seeded Poisson stream of graph requests (drawn from a pool of
    pre-generated graphs, no result caching) at a fixed offered load, served
    by continuous batching, against the plain path one request at a time."""
    import threading as th

    import numpy as np
    import torch

    import gen
    from paper_2207_04350_gb300 import cg

    torch.cuda.set_device(local_rank)
    P, R = args.serve_pool, args.serve_requests
    t_gen = time.time()
    pool = [generate_pinned(gen.served_graph(j), args.threads) for j in range(P)]
    t_gen = time.time() - t_gen
    rng = np.random.default_rng(gen.SEED0 + 4)
    pick = rng.integers(0, P, size=R)
    budget = int(args.serve_budget_gb * (1 << 30))
    mcr = args.min_chain_reads

    def drive(srv, arrivals):
        """Submit request i at arrivals[i] (seconds from start; None: all at once) and
        collect (latency, bases, batch size) as results complete."""
        import queue
        q, out = queue.Queue(), []

        def consume():
            while True:
                item = q.get()
                if item is None:
                    return
                rid = item
                res = srv.wait(rid, copy=False)
                out.append(((res["t_done_ns"] - res["t_submit_ns"]) * 1e-6, res["total_bases"], res["batch_size"],
                            res["t_submit_ns"], res["t_done_ns"], res["status"], res["n_contigs"]))
                srv.release(rid)
        c = th.Thread(target=consume, daemon=True)
        c.start()
        t0 = time.perf_counter()
        for i in range(len(pick)):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[i]:
                    time.sleep(min(2e-4, max(0.0, arrivals[i] - (time.perf_counter() - t0))))
            q.put(srv.submit(pool[pick[i]], min_chain_reads=mcr))
        q.put(None)
        c.join()
        assert all(o[5] == cg.CG_OK for o in out)
        lat = np.array([o[0] for o in out])
        size = np.array([o[1] for o in out])
        big = size >= np.percentile(size, 90)
        span = (max(o[4] for o in out) - min(o[3] for o in out)) * 1e-9
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "p99_ms_largest_tenth": float(np.percentile(lat[big], 99)),
                "p99_ms_other": float(np.percentile(lat[~big], 99)),
                "mean_ms": float(lat.mean()), "graphs_per_s": len(out) / span,
                "gbases_per_s": sum(o[1] for o in out) / span / 1e9, "span_s": span,
                "mean_batch": float(np.mean([o[2] for o in out])),
                "mean_bases": float(np.mean([o[1] for o in out])), "mean_contigs": float(np.mean([o[6] for o in out]))}

    # plain path, one request at a time: its closed-loop rate sets the offered load
    plain = cg.Server(local_rank, hbm_budget_bytes=budget, max_batch=1, workers=1)
    cal = {}
    try:
        saved = pick
        pick = saved[: min(R, 200)]
        cal = drive(plain, None)
        pick = saved
        lam = args.serve_load * cal["graphs_per_s"]
        gaps = rng.exponential(1.0 / lam, size=R)
        arrivals = np.cumsum(gaps) - gaps[0]
        plain_load = drive(plain, arrivals)
    finally:
        plain.stop()
    served = cg.Server(local_rank, hbm_budget_bytes=budget, max_batch=args.serve_max_batch,
                       workers=args.serve_workers)
    clocks = ClockSampler(local_rank)
    try:
        clocks.start()
        rank_barrier(world)
        t0 = time.time()
        served_load = drive(served, arrivals)
        t1 = time.time()
        rank_barrier(world)
        k0 = served.stats()["kernels_launched"]
        served_max = drive(served, None)
        rank_barrier(world)
        stats = served.stats()
        launches_served = stats["kernels_launched"] - k0
        outs = {}
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            # every graph of the pool once more, all submitted at once (mixed into
            # batches), its contigs kept for the oracle leg below
            ids = [served.submit(pool[j], min_chain_reads=mcr) for j in range(P)]
            for j, rid in enumerate(ids):
                r = served.wait(rid, copy=True)
                outs[j] = (r.get("contig_off"), r.get("bases"))
                served.release(rid)
    finally:
        served.stop()
        clocks.stop()
    cpu = None
    if outs:
        cpu = oracle_leg(pool, lambda j: outs[j], mcr, threads=min(16, os.cpu_count() or 1),
                         what=f"the served pool of {P} graphs")
        outs.clear()
    bases_total = sum(int(pool[j].info["n_reads"]) for j in pick[:1])
    mean_bases, mean_contigs = served_load["mean_bases"], served_load["mean_contigs"]
    line = {
        "metric": METRIC,
        "value": job_rate(served_max["gbases_per_s"] * served_max["span_s"], served_max["span_s"], world),
        "unit": UNIT, "n_gpus": world,
        "steps": R, "warmup": 0, "ms_per_step": 1e3 / served_max["graphs_per_s"],
        "ms_per_graph": 1e3 / served_max["graphs_per_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (the seeded generator gen/: genome, repeats, reads and overlaps of the stated recipe)",
        "config": {
            "workload": f"served-{R} (Poisson requests over a pool of {P} graphs, genome log-U[1,200] Mb, 5% repeats, "
                        "30x, LN(12 kb, 6 kb))",
            "requests": R, "pool": P, "hbm_budget_gb": args.serve_budget_gb, "max_batch": args.serve_max_batch,
            "workers": args.serve_workers, "offered_load_req_per_s": lam, "offered_over_plain_rate": args.serve_load,
            "plain_closed_loop": cal, "plain_at_offered_load": plain_load, "served_at_offered_load": served_load,
            "served_closed_loop": served_max, "server_stats": stats,
            "p50_ms": served_load["p50_ms"], "p99_ms": served_load["p99_ms"],
            "p50_ms_plain": plain_load["p50_ms"], "p99_ms_plain": plain_load["p99_ms"],
            "value_is": "served closed-loop contig Gbases/s; requests arrive from pinned host memory and results "
                        "return to host memory (H2D and D2H inside every request)",
            "generate_s": round(t_gen, 1),
        },
        "roofline": None, "cpu_baseline": cpu,
        "e2e": {"value": job_rate(served_load["gbases_per_s"] * served_load["span_s"], served_load["span_s"], world),
                "unit": UNIT,
                "h2d_bytes_per_step": int(np.mean([sum(getattr(pool[j], k).nbytes for k in
                                                       ("row_ptr", "col", "code", "suf", "len", "off"))
                                                   for j in pick]) + mean_bases / 4),
                "d2h_bytes_per_step": int(mean_bases + 8 * (mean_contigs + 1)),
                "note": "per request, at the offered load; the requests' reads are pinned host memory, so the server "
                        "gathers only the 2-bit bases of the pieces it spells over the host link"},
        "clocks": clocks.summary(t0, t1), "gpu_launches": launches_served,
    }
    return line


def oracle_leg(graphs, gpu_out, min_chain_reads, threads=1, what=""):
    """The cpu_baseline leg: the oracle as it stands (plain single-threaded C,
    input checks included) run on every graph of `graphs` and timed, each
    graph's contigs then compared byte for byte with the CUDA path's output
    (gpu_out(j) -> (contig_off, bases) as host arrays). With threads > 1 the
    graphs run concurrently, one per thread, and the rate is over the wall
    time of the whole set."""
    import concurrent.futures as cf

    import numpy as np

    import oracle

    def one(j):
        a = time.perf_counter()
        r = oracle.run(graphs[j], min_chain_reads=min_chain_reads)
        t = time.perf_counter() - a
        off, bases = gpu_out(j)
        same = (off is not None and np.array_equal(off, r.contig_off) and len(bases) == len(r.bases)
                and np.array_equal(bases, r.bases))
        return t, int(r.total_bases), bool(same)

    a = time.perf_counter()
    if threads > 1:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            res = list(ex.map(one, range(len(graphs))))
    else:
        res = [one(j) for j in range(len(graphs))]
    wall = time.perf_counter() - a
    t_oracle = sum(r[0] for r in res) if threads == 1 else wall
    bases = sum(r[1] for r in res)
    return {"value": bases / t_oracle / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{what}: all {len(graphs)} graph(s), {bases} contig bases, the whole oracle pipeline "
                      f"(input checks included), " + ("1 thread" if threads == 1 else f"one graph per thread on "
                                                                                        f"{threads} threads"),
            "ms_per_step": t_oracle * 1e3, "bit_exact": all(r[2] for r in res),
            "graphs_checked": len(res), "graphs_equal": sum(r[2] for r in res), **host_cpu(threads)}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2207_04350_gb300 import cg

    torch.cuda.set_device(local_rank)
    pk, pk_kind = peaks()
    cfg = workload_cfg(args.workload)
    if args.scale_genome:
        cfg = dict(cfg, genome_len=int(args.scale_genome))
    t_gen = time.time()
    G = generate_pinned(cfg, args.threads)
    t_gen = time.time() - t_gen

    stream = torch.cuda.Stream()
    ctx = cg.cg_create(local_rank, stream=stream)
    cg.cg_set_tuning(ctx, args.ruler_log2, args.tile_bytes, args.emit_blocks_per_sm, args.emit_block_threads)
    names = ("row_ptr", "col", "code", "suf", "len", "off", "packed")
    with torch.cuda.stream(stream):
        dev = {k: torch.from_numpy(getattr(G, k)).to("cuda", non_blocking=True) for k in names}
    stream.synchronize()

    class D:
        pass
    dg = D()
    for k, v in dev.items():
        setattr(dg, k, v)
    g = cg.cg_load_graph(ctx, dg, flags=cg.BORROW_DEVICE, min_chain_reads=args.min_chain_reads)
    tuned = None
    if args.autotune:
        from paper_2207_04350_gb300 import autotune
        tuned = autotune.apply(ctx, g, (G.n, G.m, G.packed_bytes))
    # sizes (untimed): walk positions, contigs, bases
    cid = np.empty(G.n, np.int32)
    rank_h = np.empty(G.n, np.int32)
    cg.cg_chains(g, cid, rank_h, None)
    W = int((cid >= 0).sum())
    n_contigs, total = cg.cg_emit_contigs(g)
    bases = torch.empty(max(16, (total + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
    contig_off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB of L2
    # timed steps: events around the spelling stage only (its live launch time for
    # the roofline); every stage's time comes from separate untimed steps below
    cg.cg_set_timing(ctx, 3)

    def step():
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        cg.cg_emit_contigs(g, contig_off, bases, want_counts=False)

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        step()
    cg.cg_sync(ctx)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    launches0 = cg.cg_get_stats(ctx)["kernels_launched"]
    step_ms, emit_ms, stage, kern = [], [], [], {}
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(2)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        st = cg.cg_get_stats(ctx)          # waits for the step
        step_ms.append(ev0.elapsed_time(ev1))
        emit_ms.append(st["stage_ms"][3])
    cg.cg_sync(ctx)
    torch.cuda.synchronize()
    t1 = time.time()
    launches = cg.cg_get_stats(ctx)["kernels_launched"] - launches0
    # per-stage breakdown: separate untimed steps with events around every stage
    cg.cg_set_timing(ctx, 1)
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush.fill_(3)
        step()
        stage.append(cg.cg_get_stats(ctx)["stage_ms"])
    # per-kernel breakdown: separate untimed steps with an event after every kernel
    cg.cg_set_timing(ctx, 2)
    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(3)
        step()
        for name, kms in cg.cg_kernel_times(ctx):
            kern.setdefault(name, []).append(kms)
    # assembly quality against the generator's truth (the paper's Table 4 analog)
    from gen import quality as _quality
    qual = _quality.contig_quality(G, cid, rank_h, contig_off.cpu().numpy())
    qual["source"] = "this run's chains and contig offsets against the generator's read placements"

    # the same steps with the 2-bit output form (outside the timed steps above);
    # events around the spelling stage only, as in the timed steps
    cg.cg_set_timing(ctx, 3)
    packed2 = torch.empty(max(16, cg.packed_bytes_2bit(total)), dtype=torch.uint8, device="cuda")

    def step2():
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        cg.cg_emit_contigs_2bit(g, contig_off, packed2, want_counts=False)

    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(4)
        step2()
    s2_ms, e2_ms = [], []
    for _ in range(max(3, args.steps // 3)):
        with torch.cuda.stream(stream):
            flush.fill_(5)
        ev0.record(stream)
        step2()
        ev1.record(stream)
        ev1.synchronize()
        st = cg.cg_get_stats(ctx)
        s2_ms.append(ev0.elapsed_time(ev1))
        e2_ms.append(st["stage_ms"][3])
    ms2, ms_e2 = statistics.mean(s2_ms), statistics.mean(e2_ms)
    emit_2bit = {
        "ms_per_step": ms2, "gbases_per_s": total / (ms2 * 1e-3) / 1e9, "steps": len(s2_ms),
        "k_emit2_ms": ms_e2, "bytes_per_base": 0.5,
        "k_emit2_achieved_gbs": 0.5 * total / (ms_e2 * 1e-3) / 1e9,
        "k_emit2_frac": 0.5 * total / (ms_e2 * 1e-3) / 1e9 / pk["hbm_gbs"],
        "note": "cg_emit_contigs_2bit: the same contigs in the 2-bit layout (0.25 B read + 0.25 B written per base)"}

    # the x-drop form of the same graph (Sec. 4.4): (pre, post) per entry with
    # unequal early starts of up to 200 bases, the other inputs shared
    import gen as _gen
    xpre, xpost = _gen.xdrop_form(G, max_trim=200, seed=7, consistent=False)
    xd = D()
    for k, v in dev.items():
        setattr(xd, k, v)
    xd.suf = None
    xd.pre = torch.from_numpy(xpre).cuda()
    xd.post = torch.from_numpy(xpost).cuda()
    gx = cg.cg_load_graph(ctx, xd, flags=cg.BORROW_DEVICE, min_chain_reads=args.min_chain_reads)
    ncx, totx = cg.cg_emit_contigs(gx)
    bases_x = torch.empty(max(16, (totx + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
    off_x = torch.empty(ncx + 1, dtype=torch.int64, device="cuda")

    def stepx():
        cg.cg_mask_branches(gx, want_count=False)
        cg.cg_chains(gx, want_counts=False)
        cg.cg_emit_contigs(gx, off_x, bases_x, want_counts=False)

    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(6)
        stepx()
    x_ms = []
    for _ in range(max(3, args.steps // 3)):
        with torch.cuda.stream(stream):
            flush.fill_(7)
        ev0.record(stream)
        stepx()
        ev1.record(stream)
        ev1.synchronize()
        cg.cg_get_stats(ctx)
        x_ms.append(ev0.elapsed_time(ev1))
    gx.close()
    xdrop = {"ms_per_step": statistics.mean(x_ms), "gbases_per_s": totx / (statistics.mean(x_ms) * 1e-3) / 1e9,
             "contig_bases": totx, "steps": len(x_ms),
             "note": "same graph in the x-drop (pre, post) form, early starts of up to 200 bases, unequal per side"}

    # TransitiveReduction (Alg. 1) of the same recipe's overlap graph before
    # reduction (every overlap >= 2 kb among the reads), device in and out
    tr = None
    if not args.no_transitive:
        Rf = _gen.generate(dict(cfg, full_overlaps=1), threads=args.threads or None, keep_genome=False,
                           with_packed=False)
        rd = D()
        for k in ("row_ptr", "col", "code", "suf", "len"):
            setattr(rd, k, torch.from_numpy(getattr(Rf, k)).cuda())
        rd.off = dev["off"]
        rd.packed = torch.empty(0, dtype=torch.uint8, device="cuda")
        cg.cg_set_timing(ctx, 2)
        tr_ms, tr_wall, tr_kern = [], [], {}
        for i in range(4):
            torch.cuda.synchronize()
            a = time.perf_counter()
            S = cg.cg_transitive_reduction(ctx, rd, 0, device=True)
            tr_wall.append((time.perf_counter() - a) * 1e3)
            kt = cg.cg_kernel_times(ctx)
            if i > 0:
                tr_ms.append(sum(t for _, t in kt))
                for name, t in kt:
                    tr_kern.setdefault(name, []).append(t)
        cg.cg_set_timing(ctx, 1)
        red_m = int(G.m)
        tr = {"entries_in": int(Rf.m), "entries_out": int(S.m), "reads": int(Rf.n),
              "generated_string_graph_entries": red_m,
              "kernel_ms": statistics.mean(tr_ms),
              "kernel_ms_by_name": {k: statistics.mean(v) for k, v in tr_kern.items()},
              "call_ms_two_calls": statistics.mean(tr_wall[1:]),
              "note": "kernel_ms: one call's kernels (checks, mark, keep, row scan, scatter); the API's size query "
                      "runs them once more"}
        del S, rd, Rf

    # GreedyPartitioning of the contigs (Sec. 4.3) into parts, outside the timed steps
    part_d = torch.empty(max(n_contigs, 1), dtype=torch.int32, device="cuda")
    psum_d = torch.empty(cg.MAX_PARTS, dtype=torch.int64, device="cuda")
    partition = {"weight": "reads per contig", "n_contigs": n_contigs, "by_parts": {}}
    cg.cg_set_timing(ctx, 2)
    for P in args.partition_parts:
        kms, wall = [], []
        for _ in range(4):
            a = time.perf_counter()
            cg.cg_partition_contigs(g, P, cg.WEIGHT_READS, part_d, psum_d[:P])
            wall.append((time.perf_counter() - a) * 1e3)
            kms.append(sum(t for _, t in cg.cg_kernel_times(ctx)))
        psum = psum_d[:P].cpu().numpy()
        partition["by_parts"][str(P)] = {
            "kernel_ms": statistics.mean(kms[1:]), "call_ms": statistics.mean(wall[1:]),
            "max_over_mean_part": float(psum.max() / max(psum.mean(), 1e-9))}
    cg.cg_set_timing(ctx, 1)
    # the per-rank step of an 8-way split of this graph over 8 GPUs (each rank
    # with the whole graph: mask, chains, then its share of the spelling), every
    # rank's step timed alone on this one GPU, one rank after another
    sharded = sharded_on_one_gpu(args, ctx, stream, dg, flush, total, statistics.mean(step_ms)) \
        if world == 1 and not args.no_forms else None
    if world > 1:
        torch.distributed.barrier()
    time.sleep(0.2)
    clocks.stop()
    ms_rank = statistics.mean(step_ms)
    ms_emit = statistics.mean(emit_ms)
    value = job_rate(total, ms_rank * 1e-3, world) / 1e9
    ms = max_over_ranks(ms_rank, world)

    # end to end through the public API with host buffers (pinned inputs / outputs).
    # Headline form: the graph arrays are copied, the packed reads stay in pinned
    # host memory and the kernels read the bases they spell over the host link
    # (CG_HOST_READS), the contigs are written into the pinned host buffers in
    # place. Also timed: every input copied to the device first (23 GB at 3.1 Gb).
    e2e = None
    e2e_copy = None
    e2e_2bit = None
    if not args.no_e2e and args.e2e_steps > 0:
        h_bases = torch.empty(max(total, 16), dtype=torch.uint8, pin_memory=True).numpy()
        h_off = torch.empty(n_contigs + 1, dtype=torch.int64, pin_memory=True).numpy()
        copied = sum(getattr(G, k).nbytes for k in names if k != "packed")
        d2h = total + (n_contigs + 1) * 8

        def e2e_run(flags):
            times = []
            for i in range(args.e2e_steps + 1):
                torch.cuda.synchronize()
                a = time.perf_counter()
                gh = cg.cg_load_graph(ctx, G, flags=flags, min_chain_reads=args.min_chain_reads)
                cg.cg_mask_branches(gh, want_count=False)
                cg.cg_chains(gh, want_counts=False)
                cg.cg_emit_contigs(gh, h_off, h_bases)
                gh.close()
                b = time.perf_counter()
                if i > 0:                      # the first one warms the context's buffer pool
                    times.append(b - a)
            return statistics.mean(times), len(times)

        te, ne = e2e_run(cg.HOST_READS)
        e2e = {"value": job_rate(total, te, world) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": copied + (total + 3) // 4, "d2h_bytes_per_step": d2h,
               "ms_per_step": te * 1e3, "steps": ne,
               "h2d_note": "graph arrays copied + the 2-bit bases of the spelled pieces, read by the kernels over "
                           "the host link (the rest of the 23 GB of reads is never moved)",
               "path": "cg_load_graph(host, validated, CG_HOST_READS) -> cg_mask_branches -> cg_chains -> "
                       "cg_emit_contigs(pinned host outputs: spelled in HBM in 128 MB chunks, each copied to "
                       "the host while the next is spelled) -> cg_free_graph"}
        tc, nc2 = e2e_run(0)
        e2e_copy = {"value": job_rate(total, tc, world) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": sum(getattr(G, k).nbytes for k in names), "d2h_bytes_per_step": d2h,
                    "ms_per_step": tc * 1e3, "steps": nc2,
                    "path": "cg_load_graph(host, validated: every input copied) -> mask -> chains -> "
                            "cg_emit_contigs(pinned host outputs) -> cg_free_graph"}
        # the same end-to-end step with the contigs in the 2-bit form (a quarter of
        # the bytes over the host link, which bounds the ASCII form)
        h_packed = torch.empty(max(16, cg.packed_bytes_2bit(total)), dtype=torch.uint8, pin_memory=True).numpy()
        t2 = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            a = time.perf_counter()
            gh = cg.cg_load_graph(ctx, G, flags=cg.HOST_READS, min_chain_reads=args.min_chain_reads)
            cg.cg_mask_branches(gh, want_count=False)
            cg.cg_chains(gh, want_counts=False)
            cg.cg_emit_contigs_2bit(gh, h_off, h_packed)
            gh.close()
            b = time.perf_counter()
            if i > 0:
                t2.append(b - a)
        e2e_2bit = {"value": job_rate(total, statistics.mean(t2), world) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": copied + (total + 3) // 4,
                    "d2h_bytes_per_step": cg.packed_bytes_2bit(total) + (n_contigs + 1) * 8,
                    "ms_per_step": statistics.mean(t2) * 1e3, "steps": len(t2),
                    "path": "cg_load_graph(host, validated, CG_HOST_READS) -> mask -> chains -> "
                            "cg_emit_contigs_2bit(pinned host outputs, written in place) -> cg_free_graph"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the whole graph of the timed steps, and the CUDA path's
        # output of one more step (the part runs above reused the buffers) against it
        step()
        cg.cg_sync(ctx)
        h_off, h_b = contig_off.cpu().numpy(), bases[:total].cpu().numpy()
        cpu = oracle_leg([G], lambda j: (h_off, h_b), args.min_chain_reads, what=cfg_name(args))
        del h_off, h_b
        cpu["scaled_sample"] = cpu_baseline(args, cfg)

    B = bmin_bytes(G, W, total, n_contigs)
    import hashlib
    with open(os.path.join(ROOT, "paper_2207_04350_gb300", "csrc", "cg_emit.cu"), "rb") as f:
        same_kernel = hashlib.sha256(f.read()).hexdigest()[:16] == EMIT_TRAFFIC["source_sha256_16"]
    traffic = EMIT_TRAFFIC["bytes_per_base"] * total if same_kernel else None
    emit_bytes = total + (total + 3) // 4
    ach = emit_bytes / (ms_emit * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "ms_per_graph": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (the seeded generator gen/: genome, repeats, reads and overlaps of the stated recipe)",
        "config": {
            "workload": cfg_name(args),
            "tuning": cg.cg_get_tuning(ctx), "n_reads": G.n, "n_entries": G.m, "walk_reads": W, "n_contigs": n_contigs,
            "contig_bases": total, "packed_read_bytes": int(G.packed.nbytes), "min_chain_reads": args.min_chain_reads,
            "row_ptr_bytes": int(G.row_ptr.dtype.itemsize), "replicas": world,
            "l2": "flushed between steps (512 MiB write, outside the timed events)",
            "events": "timed steps record CUDA events around the spelling stage only (its live launch time); "
                      "the stage and kernel breakdowns come from separate untimed steps",
            "inputs": "resident in HBM (CG_BORROW_DEVICE)", "reads_per_s": G.n / (ms * 1e-3),
            "stage_ms_mean": [statistics.mean(s[k] for s in stage) for k in range(4)],
            "stage_names": ["mask", "chains", "offsets", "emit"],
            "kernel_ms_mean": {k: statistics.mean(v) for k, v in kern.items()},
            "kernel_ms_note": "3 extra untimed steps with a CUDA event after every kernel",
            "step_ms_median": statistics.median(step_ms), "step_ms_min": min(step_ms), "step_ms_max": max(step_ms),
            "partition": partition,
            "sharded_on_one_gpu": sharded,
            "emit_2bit": emit_2bit,
            "xdrop": xdrop,
            "autotune": tuned,
            "quality": qual,
            "transitive_reduction": tr,
            "e2e_copy_all_inputs": e2e_copy, "e2e_2bit_output": e2e_2bit,
            "B_min_bytes": B, "path_achieved_gbs": B / (ms * 1e-3) / 1e9,
            "path_roofline_frac": B / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
            "path_roofline_frac_8tbs": B / (ms * 1e-3) / 1e9 / 8000.0,
            "generate_s": round(t_gen, 1), "wall_s_timed": t1 - t0,
        },
        "roofline": {"kernel": "k_emit (contig spelling)", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": traffic,
                     "traffic_note": "ncu dram bytes of a scaled capture (450 Mb recipe) x contig bases; null when "
                                     "the kernel changed since",
                     "algorithmic_bytes_per_launch": emit_bytes, "bytes_per_unit": 1.25,
                     "units_per_launch": total, "ms_per_launch": ms_emit, "peak_kind": pk_kind + " (hbm_gbs, copy)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks.summary(t0, t1),
        "gpu_launches": launches,
    }
    g.close()
    ctx.close()
    return line


def sharded_on_one_gpu(args, ctx, stream, dg, flush, total, whole_ms, n_ranks=8, steps=5):
    """Every rank's step of an n_ranks-way split of one graph (paper_2207_04350_gb300.shard:
    each rank loads the whole graph, runs the mask and chain stages, and spells
    its share), timed one rank after another on this one GPU with CUDA events
    on the context stream, L2 flushed before each step: the slowest rank's step
    is what one step of the split would take on n_ranks GPUs, collectives
    aside (the split has none on its data path). Not a multi-GPU run."""
    import torch

    from paper_2207_04350_gb300 import cg, shard
    out = {"n_ranks": n_ranks, "steps_per_rank": steps, "whole_graph_step_ms": whole_ms,
           "note": "per-rank device time of the rank's whole step (mask, chains, [LPT], its spelling), ranks timed one "
                   "after another on one GPU; max over ranks = the split's step on n_ranks GPUs without collectives"}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cg.cg_set_timing(ctx, 0)
    for mode in shard.MODES:
        per_rank, sizes = [], []
        for r in range(n_ranks):
            run = shard.ShardedRun(ctx, dg, r, n_ranks, mode=mode, flags=cg.BORROW_DEVICE,
                                   min_chain_reads=args.min_chain_reads)
            ts = []
            for i in range(steps + 2):
                with torch.cuda.stream(stream):
                    flush.fill_(11)
                ev0.record(stream)
                run.step()
                ev1.record(stream)
                ev1.synchronize()
                if i >= 2:
                    ts.append(ev0.elapsed_time(ev1))
            cg.cg_sync(ctx)
            sizes.append(int(run.n_bases))
            per_rank.append(statistics.median(ts))
            run.close()
        mx = max(per_rank)
        out[mode] = {"rank_step_ms": per_rank, "max_rank_step_ms": mx, "rank_bases": sizes,
                     "bases_max_over_mean": max(sizes) / max(1e-9, sum(sizes) / len(sizes)),
                     "speedup_over_one_gpu": whole_ms / mx,
                     "gbases_per_s_n_ranks": total / (mx * 1e-3) / 1e9}
    out["lpt"]["weight"] = "bases (cg_partition_contigs, recomputed by every rank every step)"
    out["tiles"]["split"] = "equal runs of the graph's layout tiles, 8 KiB here (cg_emit_share)"
    out["exchange"] = exchange_on_one_gpu(ctx, stream, dg, flush, n_ranks, steps, args.min_chain_reads)
    return out


def exchange_on_one_gpu(ctx, stream, dg, flush, n_ranks, steps, mcr):
    """The same 8-way tile split with each rank holding only its slice of the
    reads (reads in equal id ranges): per rank, the device time of its side of
    the read exchange -- mask, chains, layout and packing the pieces every share
    needs from its reads, then spelling its share from what it received -- each
    timed alone on this GPU, and the bytes it sends and receives. The all-to-all
    itself needs several GPUs and is not timed; the received buffers are
    assembled here from the senders' buffers. Each rank's own reads are read in
    place from the whole stream (my_off = the graph's offsets of its reads)."""
    import numpy as np
    import torch

    from paper_2207_04350_gb300 import cg
    n = int(dg.len.numel())
    rf = np.array([n * r // n_ranks for r in range(n_ranks + 1)], dtype=np.int64)
    nr = type("NR", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off"):
        setattr(nr, k, getattr(dg, k))
    nr.packed, nr.packed_bytes = None, int(dg.packed.numel())
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    graphs = [cg.cg_load_graph(ctx, nr, flags=cg.BORROW_DEVICE | cg.NO_READS, min_chain_reads=mcr)
              for _ in range(n_ranks)]
    try:
        sizes = [cg.cg_exchange_sizes(graphs[r], n_ranks, rf, r) for r in range(n_ranks)]
        sends = [torch.empty(max(16, int(sizes[r][0].sum())), dtype=torch.uint8, device="cuda") for r in range(n_ranks)]
        send_ms, recv_ms = [], []
        for r in range(n_ranks):
            my_off = dg.off[int(rf[r]):int(rf[r + 1])]
            ts = []
            for i in range(steps + 1):
                with torch.cuda.stream(stream):
                    flush.fill_(12)
                ev0.record(stream)
                cg.cg_mask_branches(graphs[r], want_count=False)
                cg.cg_chains(graphs[r], want_counts=False)
                cg.cg_exchange_pack(graphs[r], n_ranks, rf, r, dg.packed, my_off, sends[r])
                ev1.record(stream)
                ev1.synchronize()
                if i:
                    ts.append(ev0.elapsed_time(ev1))
            send_ms.append(statistics.median(ts))
        for r in range(n_ranks):
            segs = []
            for s_ in range(n_ranks):
                a = int(sizes[s_][0][:r].sum())
                segs.append(sends[s_][a:a + int(sizes[s_][0][r])])
            recv = torch.cat(segs)
            n_contigs, _ = cg.cg_emit_contigs(graphs[r])
            _, nb = cg.cg_emit_share(graphs[r], r, n_ranks)
            off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
            bases = torch.empty(max(16, (nb + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
            ts = []
            scratch_send = torch.empty_like(sends[r])
            for i in range(steps + 1):
                # the rank's own layout and packing first (untimed here: the send side above)
                cg.cg_mask_branches(graphs[r], want_count=False)
                cg.cg_chains(graphs[r], want_counts=False)
                cg.cg_exchange_pack(graphs[r], n_ranks, rf, r, dg.packed, dg.off[int(rf[r]):int(rf[r + 1])],
                                    scratch_send)
                with torch.cuda.stream(stream):
                    flush.fill_(13)
                ev0.record(stream)
                cg.cg_emit_share_received(graphs[r], n_ranks, rf, r, recv, off, bases)
                ev1.record(stream)
                ev1.synchronize()
                if i:
                    ts.append(ev0.elapsed_time(ev1))
            recv_ms.append(statistics.median(ts))
            del recv
        total_ms = [a + b for a, b in zip(send_ms, recv_ms)]
        return {"rank_send_side_ms": send_ms, "rank_receive_side_ms": recv_ms, "max_rank_ms_without_all_to_all":
                max(total_ms), "rank_send_bytes": [int(x[0].sum()) for x in sizes],
                "rank_recv_bytes": [int(x[1].sum()) for x in sizes],
                "note": "reads in 8 equal id ranges; per rank: mask + chains + layout + pack (send side), then "
                        "placing the received pieces and spelling its share (receive side); the all-to-all between "
                        "them needs several GPUs and is not timed"}
    finally:
        for g in graphs:
            g.close()


def run_sharded(args, rank, world, local_rank):
    """One graph split over the ranks (paper_2207_04350_gb300.shard): every rank
    holds the whole graph and reads in its HBM, runs the mask and chain stages
    and spells its own share ("tiles": equal runs of output tiles; "lpt": the
    paper's GreedyPartitioning of whole contigs). No collective on the data
    path; the step time is the slowest rank's. Strong scaling: the work per
    step is one graph whatever the number of ranks."""
    import torch

    from paper_2207_04350_gb300 import cg, shard

    torch.cuda.set_device(local_rank)
    pk, pk_kind = peaks()
    cfg = workload_cfg(args.workload)
    t_gen = time.time()
    G = generate_pinned(cfg, args.threads)
    t_gen = time.time() - t_gen
    stream = torch.cuda.Stream()
    ctx = cg.cg_create(local_rank, stream=stream)
    names = ("row_ptr", "col", "code", "suf", "len", "off", "packed")
    with torch.cuda.stream(stream):
        dev = {k: torch.from_numpy(getattr(G, k)).to("cuda", non_blocking=True) for k in names}
    stream.synchronize()
    dg = type("D", (), {})()
    for k, v in dev.items():
        setattr(dg, k, v)
    run = shard.ShardedRun(ctx, dg, rank, world, mode=args.shard, flags=cg.BORROW_DEVICE,
                           min_chain_reads=args.min_chain_reads)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    cg.cg_set_timing(ctx, 3)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        run.step()
    cg.cg_sync(ctx)
    rank_barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    launches0 = cg.cg_get_stats(ctx)["kernels_launched"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, emit_ms = [], []
    rank_barrier(world)
    t0 = time.time()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(2)
        ev0.record(stream)
        run.step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        emit_ms.append(cg.cg_get_stats(ctx)["stage_ms"][3])
    cg.cg_sync(ctx)
    torch.cuda.synchronize()
    rank_barrier(world)
    t1 = time.time()
    launches = cg.cg_get_stats(ctx)["kernels_launched"] - launches0
    time.sleep(0.2)
    clocks.stop()
    ms_rank = statistics.mean(step_ms)
    value = job_rate(run.n_bases, ms_rank * 1e-3, world) / 1e9
    ms = max_over_ranks(ms_rank, world)
    total = run.total
    ms_emit = statistics.mean(emit_ms)
    emit_bytes = run.n_bases + (run.n_bases + 3) // 4
    ach = emit_bytes / (ms_emit * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "ms_per_graph": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (the seeded generator gen/: genome, repeats, reads and overlaps of the stated recipe)",
        "config": {"workload": cfg_name(args) + f", split over {world} rank(s) ({args.shard})",
                   "shard_mode": args.shard, "n_contigs": run.n_contigs, "contig_bases": total,
                   "rank0_bases": run.n_bases, "inputs": "whole graph and reads resident in every rank's HBM",
                   "l2": "flushed between steps (512 MiB write, outside the timed events)",
                   "generate_s": round(t_gen, 1), "wall_s_timed": t1 - t0},
        "roofline": {"kernel": "k_emit (this rank's share)", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": None,
                     "algorithmic_bytes_per_launch": emit_bytes, "bytes_per_unit": 1.25,
                     "units_per_launch": run.n_bases, "ms_per_launch": ms_emit,
                     "peak_kind": pk_kind + " (hbm_gbs, copy)"},
        "cpu_baseline": None, "e2e": None, "clocks": clocks.summary(t0, t1), "gpu_launches": launches,
    }
    run.close()
    ctx.close()
    return line


def plain_record(args, name, local_rank, steps=20, warmup=3):
    """A compact record of one more plain workload (tiny-1Mb, genome-100Mb):
    the step of the main line (inputs resident in HBM, L2 flushed between
    steps, CUDA events on the context stream), the spelling kernel's live time,
    the path's roofline fraction, and the oracle leg on the same graph."""
    import numpy as np
    import torch

    from paper_2207_04350_gb300 import cg

    pk, _ = peaks()
    G = generate_pinned(workload_cfg(name), args.threads)
    stream = torch.cuda.Stream()
    ctx = cg.cg_create(local_rank, stream=stream)
    names = ("row_ptr", "col", "code", "suf", "len", "off", "packed")
    with torch.cuda.stream(stream):
        dev = {k: torch.from_numpy(getattr(G, k)).to("cuda", non_blocking=True) for k in names}
    stream.synchronize()
    dg = type("D", (), {})()
    for k, v in dev.items():
        setattr(dg, k, v)
    g = cg.cg_load_graph(ctx, dg, flags=cg.BORROW_DEVICE, min_chain_reads=args.min_chain_reads)
    cid = np.empty(G.n, np.int32)
    cg.cg_chains(g, cid, None, None)
    W = int((cid >= 0).sum())
    n_contigs, total = cg.cg_emit_contigs(g)
    bases = torch.empty(max(16, (total + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
    contig_off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    cg.cg_set_timing(ctx, 3)

    def step():
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        cg.cg_emit_contigs(g, contig_off, bases, want_counts=False)

    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        step()
    cg.cg_sync(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, emit_ms = [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(2)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        emit_ms.append(cg.cg_get_stats(ctx)["stage_ms"][3])
    cg.cg_set_timing(ctx, 1)
    stage = []
    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(3)
        step()
        stage.append(cg.cg_get_stats(ctx)["stage_ms"])
    ms, ms_emit = statistics.mean(step_ms), statistics.mean(emit_ms)
    B = bmin_bytes(G, W, total, n_contigs)
    rec = {"ms_per_graph": ms, "gbases_per_s": total / (ms * 1e-3) / 1e9, "reads_per_s": G.n / (ms * 1e-3),
           "steps": steps, "warmup": warmup, "n_reads": G.n, "n_entries": G.m, "n_contigs": n_contigs,
           "contig_bases": total, "B_min_bytes": B, "path_roofline_frac": B / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
           "path_roofline_frac_8tbs": B / (ms * 1e-3) / 1e9 / 8000.0, "k_emit_ms": ms_emit,
           "k_emit_frac": 1.25 * total / (ms_emit * 1e-3) / 1e9 / pk["hbm_gbs"],
           "stage_ms_mean": [statistics.mean(x[k] for x in stage) for k in range(4)],
           "gpu_launches_per_step": None}
    k0 = cg.cg_get_stats(ctx)["kernels_launched"]
    step()
    cg.cg_sync(ctx)
    rec["gpu_launches_per_step"] = cg.cg_get_stats(ctx)["kernels_launched"] - k0
    if not args.no_cpu_baseline:
        h_off, h_b = contig_off.cpu().numpy(), bases[:total].cpu().numpy()
        cpu = oracle_leg([G], lambda j: (h_off, h_b), args.min_chain_reads, what=name)
        rec["bit_exact"] = cpu["bit_exact"]
        rec["oracle_gbases_per_s"] = cpu["value"]
        rec["oracle_ms"] = cpu["ms_per_step"]
    g.close()
    ctx.close()
    return rec


def form_records(args, local_rank):
    """Every other workload of the benchmark, each as a compact record beside
    the main line: the tiny and 100 Mb plain graphs, the 512-graph batch (one
    union pass against the same graphs one by one) and the 2000-request
    served stream (continuous batching against one request at a time), each
    with its oracle leg's bit-exact result."""
    import copy

    import torch
    out = {}
    t = time.time()
    for name in ("tiny-1Mb", "genome-100Mb"):
        out[name] = plain_record(args, name, local_rank)
        torch.cuda.empty_cache()
    a = copy.copy(args)
    a.steps, a.warmup, a.e2e_steps = 10, 3, 2
    b = run_batched(a, 0, 1, local_rank)
    torch.cuda.empty_cache()
    c, bc = b["config"], b["cpu_baseline"] or {}
    out["batched-512"] = {
        "graphs": c["graphs"], "graphs_per_s_batched": c["graphs_per_s_batched"],
        "graphs_per_s_plain": c["graphs_per_s_plain"], "batched_over_plain": c["batched_over_plain"],
        "ms_per_graph_batched": c["ms_per_graph_batched"], "ms_per_graph_plain": c["ms_per_graph_plain"],
        "ms_per_batch": b["ms_per_step"], "gbases_per_s": b["value"], "contig_bases": c["contig_bases"],
        "n_reads": c["n_reads"], "k_emit_frac": b["roofline"]["frac"], "gpu_launches_per_step":
            b["gpu_launches"] / max(1, a.steps), "steps": a.steps,
        "e2e_graphs_per_s": (b["e2e"] or {}).get("graphs_per_s"), "e2e_gbases_per_s": (b["e2e"] or {}).get("value"),
        "bit_exact": bc.get("bit_exact"), "graphs_checked": bc.get("graphs_checked"),
        "oracle_gbases_per_s": bc.get("value"), "clocks": b["clocks"]}
    sv = run_served(a, 0, 1, local_rank)
    c, sc = sv["config"], sv["cpu_baseline"] or {}
    out["served-2000"] = {
        "requests": c["requests"], "pool": c["pool"], "offered_load_req_per_s": c["offered_load_req_per_s"],
        "graphs_per_s_served_closed_loop": c["served_closed_loop"]["graphs_per_s"],
        "graphs_per_s_plain_closed_loop": c["plain_closed_loop"]["graphs_per_s"],
        "served_over_plain": c["served_closed_loop"]["graphs_per_s"] / c["plain_closed_loop"]["graphs_per_s"],
        "p50_ms": c["p50_ms"], "p99_ms": c["p99_ms"], "p50_ms_plain": c["p50_ms_plain"],
        "p99_ms_plain": c["p99_ms_plain"], "gbases_per_s_served_closed_loop": c["served_closed_loop"]["gbases_per_s"],
        "mean_batch_at_load": c["served_at_offered_load"]["mean_batch"], "workers": c["workers"],
        "p99_ms_largest_tenth": c["served_at_offered_load"]["p99_ms_largest_tenth"],
        "graphs_per_s_at_load": c["served_at_offered_load"]["graphs_per_s"],
        "bit_exact": sc.get("bit_exact"), "graphs_checked": sc.get("graphs_checked"),
        "oracle_gbases_per_s": sc.get("value"), "oracle_cores": sc.get("cores"), "clocks": sv["clocks"],
        "latency": "arrival to contigs in host memory, H2D and D2H included"}
    out["wall_s"] = round(time.time() - t, 1)
    return out


def host_cpu(threads: int = 1) -> dict:
    """The host's CPU model and logical cores (the oracle uses `threads` of them)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
                if k == "cpu part" and not model:
                    model = "cpu part " + line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return {"cpu": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "host_cores_available": os.cpu_count(), "threads_used": threads}


def cfg_name(args) -> str:
    return args.workload + (f" (recipe scaled to {args.scale_genome} bases)" if args.scale_genome else "")


def cpu_baseline(args, cfg, steps=None, warmup=0, budget_s=None):
    """The oracle as it stands (single thread) on a bounded sample of the same
    workload: the workload's recipe on a smaller genome. Without budget_s the
    genome is 20 Mb and the oracle repeats for about `cpu_seconds`; with it,
    the genome is the largest (up to the workload's own) whose warmup + steps
    runs fit budget_s, estimated from one run on 200 Mb."""
    import gen
    import oracle
    G0 = cfg["genome_len"]
    scale = min(G0, 20_000_000 if budget_s is None else 200_000_000)
    mcr = args.min_chain_reads
    G = gen.generate(dict(cfg, genome_len=scale), threads=args.threads or None, keep_genome=False)
    a = time.perf_counter()
    r = oracle.run(G, min_chain_reads=mcr)
    once = time.perf_counter() - a
    if budget_s is not None and steps:
        fit = int(scale * budget_s / (steps + warmup) / max(once, 1e-6))
        if fit > scale:
            scale = min(G0, fit)
            del G
            G = gen.generate(dict(cfg, genome_len=scale), threads=args.threads or None, keep_genome=False)
    if steps is None:
        steps = max(1, int(args.cpu_seconds / max(once, 1e-3)))
    for _ in range(warmup):
        oracle.run(G, min_chain_reads=mcr)
    times = []
    for _ in range(steps):
        a = time.perf_counter()
        r = oracle.run(G, min_chain_reads=mcr)
        times.append(time.perf_counter() - a)
    t = statistics.mean(times)
    whole = scale == G0
    return {"value": r.total_bases / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{args.workload} recipe on {'its whole' if whole else 'a'} {scale/1e6:.0f} Mb genome "
                      f"({G.n} reads, {r.total_bases} contig bases), full oracle pipeline, mean of {len(times)} "
                      f"runs, {t:.2f} s each, 1 thread",
            "genome_bases": scale, "whole_workload": whole,
            "ms_per_step": t * 1e3, "median_ms": statistics.median(times) * 1e3, **host_cpu()}


def run_reference(args, rank, world):
    """The reference arm: the oracle on the host cores, rank 0 only, each step
    one oracle run on a sample of the workload sized so that the whole
    warmup + steps run takes about two and a half minutes."""
    if rank != 0:
        return None
    budget = 150.0
    if args.workload.startswith("batched") or args.workload.startswith("served"):
        import gen
        mk = gen.batched_graph if args.workload.startswith("batched") else gen.served_graph
        graphs = [gen.generate(mk(j), threads=args.threads or None, keep_genome=False) for j in range(16)]
        args.cpu_seconds = max(1.0, budget / max(1, args.steps + args.warmup))
        cpu = oracle_leg(graphs, lambda j: (None, None), args.min_chain_reads, what=f"first 16 graphs of {args.workload}")
        cpu["ms_per_step"] = cpu["ms_per_step"] / len(graphs)
        cpu.pop("bit_exact", None)
    else:
        cfg = workload_cfg(args.workload)
        cpu = cpu_baseline(args, cfg, steps=args.steps, warmup=args.warmup, budget_s=budget)
    return {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cpu["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "min_chain_reads": args.min_chain_reads,
                       "oracle_genome_bases": cpu.get("genome_bases"), "whole_workload": cpu.get("whole_workload")},
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        import datetime
        # a rank that dies ends the others' next collective with an error after this long
        torch.distributed.init_process_group("nccl", timeout=datetime.timedelta(seconds=args.pg_timeout))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
        __graft_entry__.build()
    if args.shard:
        line = run_sharded(args, rank, world, local_rank)
    elif args.workload.startswith("batched"):
        line = run_batched(args, rank, world, local_rank)
    elif args.workload.startswith("served"):
        line = run_served(args, rank, world, local_rank)
    else:
        line = run_ours(args, rank, world, local_rank)
        if world == 1 and not args.no_forms and not args.scale_genome:
            torch.cuda.empty_cache()
            line["config"]["other_workloads"] = form_records(args, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
