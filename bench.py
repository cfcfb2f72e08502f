#!/usr/bin/env python
"""Benchmark of the exact multi-objective search on one GB300.

Workload (default): one start->goal query on the seeded 256x256 8-connected
3-objective ship grid (move length, length x current, length x wave; 5% land;
corner to corner). A step is the whole hot path: ideal-point heuristic, the
ordered-parallel search to the exact Pareto front, sorted front + paths, and
the device->host copy of the result.

value  = Pareto labels/s, counted as the oracle's number of labels extracted
         for this query (taken from the committed oracle fixture) divided by
         the GPU time-to-front, so labels the parallel search extracts beyond
         the sequential count earn nothing. The GPU's own extraction rate and
         the work ratio are reported beside it.
e2e    = the same metric through the C ABI with host buffers: graph upload,
         solve, result download, graph release inside the timed region.

--impl reference times the oracle (sequential NAMOA*, Algorithm 1) on the host
cores on a bounded sample of the same query (a label budget).

Other workloads (--workload):
  ship128-d3        the same recipe on a 128x128 grid: the small case used for
                    ncu captures (value = the GPU's own labels/s)
  ship256-d5-batch  1,024 start/goal pairs (Chebyshev distance 16-128) on the
                    5-objective ship grid in one continuous-batching launch;
                    value = queries/s, beside one query per launch on a sample
  road200k-d4-batch the fewest-hop queries of the 256 on the 200k-node
                    4-objective road-like graph in one launch, each under a
                    label budget; value = exact fronts per second, beside one
                    query per launch on the same queries
  serve             Poisson arrivals over the device-resident 32x32, 256x256 and
                    200k-node graphs, d ~ U{2..5} clamped, at three rates;
                    p50/p99 latency and queries/s beside one query per launch
  order             ordered (priority) against FIFO windows of the same width:
                    labels extracted, work ratio and time (Sec. 4, 7.1)

The default line also carries, as extra keys, a config-4 batch subset timed
as one launch and as one query per launch on the same queries ("batch", with
the batch kernel's roofline) and the d = 12 time-expanded route
("route_d12": time-to-front and work ratio against the oracle).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload NAME]
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

import numpy as np  # noqa: E402

import synth  # noqa: E402

FIXTURE = os.path.join(ROOT, "tests", "golden", "config2_seed1_q0.front")
METRIC = "Pareto labels/s (time-to-front per query)"
UNIT = "labels/s"
CPU_SAMPLE_LABELS = 1_500_000

# DRAM bytes (read + write) of one search_grid_kernel launch of the default
# workload, from ncu captures (profiles/search_grid_kernel_ship256-d3_dram.md),
# keyed by the digest of the kernel sources and launch options (the window
# among them) they were taken with: a launch whose digest has no entry (the
# sources changed, or another window was chosen) reports null.
TRAFFIC = {
    "7368f652d975998e": 6032931840 + 4144625152,  # W = 262144
    "903b9a5f7ee557e5": 2759832064 + 2360845056,  # W = 65536
}


# the translation unit of the search kernels: the file and every header it includes
KERNEL_SOURCES = ("paper_2411_16667_gb300/csrc/search_impl.cuh", "paper_2411_16667_gb300/csrc/search_inst.cu",
                  "paper_2411_16667_gb300/csrc/search.cuh", "paper_2411_16667_gb300/csrc/opmos_dev.cuh",
                  "include/opmos.h")


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and trailing blanks (comments do not
    change the compiled kernel)."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_source_digest(launch=(), read=None) -> str:
    """sha256 over the search kernel's sources (names and contents without
    comments) and the launch options (window, lanes per label, tile, delta):
    what the kernel's DRAM traffic on a given workload depends on."""
    import hashlib
    if read is None:
        def read(rel):
            with open(os.path.join(ROOT, rel)) as f:
                return f.read()
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(rel.encode())
        h.update(strip_comments(read(rel)).encode())
    h.update(repr(tuple(int(x) for x in launch)).encode())
    return h.hexdigest()[:16]


def fixture_stats() -> dict:
    """Oracle counters of the workload query, written by tests/golden/make_golden.py."""
    meta = {}
    with open(FIXTURE) as f:
        for line in f:
            if line.startswith("graph "):
                meta["digest"] = line.split()[2]
            elif line.startswith("stats "):
                meta.update({k: int(v) for k, v in (kv.split("=") for kv in line.split()[1:])})
            elif line.startswith("count "):
                meta["count"] = int(line.split()[1])
                break
    return meta


def oracle_count_bytes(st: dict, d: int) -> int:
    """Algorithmic bytes of the sequential oracle's own counters, with the same
    per-unit figures the device counters use: per extracted label 8d+12, per
    candidate 4+8d, per compared vector 4d, per inserted label 4d+24, per
    pruned label 4. The GPU gets no credit for the work it adds."""
    pruned = st["pruned_open"] + st["pruned_open_goal"] + st["pruned_closed"] + st["pruned_p"]
    return (st["extracted"] * (8 * d + 12) + st["candidates"] * (4 + 8 * d) + st["comparisons"] * 4 * d
            + st["inserted"] * (4 * d + 24) + pruned * 4)


def cpu_sample(g, s, t, budget=CPU_SAMPLE_LABELS) -> dict:
    """The oracle as it stands, single-threaded, on the first `budget` labels."""
    import oracle
    oracle.build()
    h = oracle.heuristic(g, t)
    res = oracle.solve(g, s, t, h=h, label_budget=budget, partial_ok=True)
    st = res.stats
    secs = st["ns"] / 1e9
    return {"value": st["extracted"] / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"sequential NAMOA* (Algorithm 1) on the same query, stopped at {budget} labels "
                      f"({st['extracted']} extracted in {secs:.2f} s main loop)"}


_CPU_GRAPH = {}


def _cpu_init(n, d, rowptr, col, cost):
    import oracle
    _CPU_GRAPH["g"] = synth.Graph("cpu-sample", n, d, rowptr, col, cost, {})
    oracle.build()


def _cpu_solve(job):
    import oracle
    s, t, budget = job
    t0 = time.perf_counter()
    f = oracle.solve(_CPU_GRAPH["g"], s, t, label_budget=budget, partial_ok=True)
    return time.perf_counter() - t0, int(f.stats["partial"])


def cpu_batch_sample(g, queries, every: int, budget: int = 0) -> dict:
    """The oracle as it stands on all host cores, one query per process
    (queries are independent), over every ``every``-th query of the batch:
    queries answered per wall second. The pool is started with spawn, so a
    CUDA context in this process is not inherited."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    sample = queries[::every]
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, len(sample)), initializer=_cpu_init,
                  initargs=(g.n, g.d, g.rowptr, g.col, g.cost)) as pool:
        t0 = time.perf_counter()
        res = pool.map(_cpu_solve, [(s, t, budget) for s, t in sample], chunksize=1)
        wall = time.perf_counter() - t0
    over = sum(p for _, p in res)
    used = min(cores, len(sample))
    busy = sum(t for t, _ in res)
    # a whole batch keeps every core busy, so its throughput is the sample's
    # queries per core-second of oracle time times the cores; the sample's own
    # wall time is bounded by its longest query
    return {"value": len(sample) * used / busy, "unit": "queries/s", "cores": used, "kind": "oracle",
            "sample": f"{len(sample)} of the {len(queries)} queries (1 in {every}), one per process, "
                      f"label budget {budget or 'none'}; {over} over budget; {busy:.1f} core-s of oracle "
                      f"time, longest query {max(t for t, _ in res):.1f} s, {wall:.1f} s wall "
                      f"({len(sample) / wall:.3g} queries per wall second)"}


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_queries(n: int, rank: int, world: int, est=None) -> list[int]:
    """Split of n independent queries over the ranks, round-robin in
    decreasing order of estimated cost (``est``; index order without one),
    so every rank gets a similar mix of long and short searches. Queries
    share nothing, so the ranks exchange no data; only the timing is
    reduced. Returns the rank's query indices in increasing order."""
    order = list(range(n)) if est is None else sorted(range(n), key=lambda i: (-est[i], i))
    return sorted(order[rank::world])


def grid_distance(g, queries) -> list[int]:
    """Chebyshev distance of each (start, goal) on a grid graph (an estimate
    of the search's cost; 1 when the graph is not a grid)."""
    cols = g.meta.get("cols")
    if not cols or g.meta.get("windows"):
        return [1] * len(queries)
    return [max(abs(s // cols - t // cols), abs(s % cols - t % cols)) for s, t in queries]


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """Maximum of x over the ranks of the default process group (x itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


ROUTES = os.path.join(ROOT, "tests", "golden", "routes.digests")
ROUTE_D12 = (1, 6, 8, 24, 12)  # seed, rows, cols, windows, d of the default line's high-d route


def route_digests() -> dict:
    """Oracle digests of the time-expanded routes (tests/golden/make_golden.py routes)."""
    out = {}
    with open(ROUTES) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, gdig, s, t, count, labels, extracted, fdig = line.split()
            out[name] = {"graph": gdig, "start": int(s), "goal": int(t), "count": int(count),
                         "labels": int(labels), "extracted": int(extracted), "front": fdig}
    return out


def front_digest(costs) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(costs, dtype="<u4").tobytes()).hexdigest()[:16]


def tuned_window(opmos, stream, g, q, windows) -> int:
    """The autotuner's single-query window for a workload, calibrated on a
    DIFFERENT instance of the same recipe (another seed) outside the timed
    region: the window that gives the fastest search there."""
    from paper_2411_16667_gb300 import autotune
    G = opmos.opmos_graph.from_synth(g)
    return autotune.autotune(G, q[:1], mode="single", windows=windows, lanes=(8,), tiles=(32,),
                             stream_ptr=stream.cuda_stream).window


def route_leg(opmos, torch, stream, steps: int, window: int = 0, flags: int = 0) -> dict:
    """The d = 12 time-expanded route (label processing dominates, Sec. 4):
    time-to-front and work ratio against the oracle's committed counters; the
    window autotuned on the route of the next seed unless given."""
    seed, rows, cols, windows, d = ROUTE_D12
    g, q = synth.time_route(seed, rows, cols, windows, d)
    ref = route_digests()[g.name]
    if ref["graph"] != g.digest():
        raise RuntimeError("regenerated route does not match its oracle digest")
    if not window:
        window = tuned_window(opmos, stream, *synth.time_route(seed + 1, rows, cols, windows, d),
                              (256, 1024, 4096))
    G = opmos.opmos_graph.from_synth(g)
    s, t = q[0]
    opt = opmos.opmos_default_options(stream=stream.cuda_stream, window=window, flags=flags)
    r = opmos.opmos_solve(G, s, t, options=opt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(max(1, steps))]
    for a, b in ev:
        a.record(stream)
        r = opmos.opmos_solve(G, s, t, options=opt)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    st = r.stats
    return {"workload": f"{g.name}: time-expanded ship route, {rows}x{cols} cells x {windows} windows, "
                        f"{g.n} nodes, {g.m} arcs, d = {d}",
            "front_size": int(r.costs.shape[0]), "front_matches_oracle": front_digest(r.costs) == ref["front"],
            "time_to_front_ms": ms, "search_kernel_ms": st["search_ns"] / 1e6, "window": window,
            "gpu_labels_extracted": st["extracted"], "oracle_labels_extracted": ref["extracted"],
            "work_ratio": st["extracted"] / ref["extracted"],
            "oracle_labels_per_s": ref["extracted"] / (ms / 1e3),
            "frontier_cmp": st["frontier_cmp"], "p_cmp": st["p_cmp"], "steps": st["steps"]}


BATCH_EVERY = 8        # the default line's batch subset: every 8th of the 1,024 config-4 queries
BATCH_WINDOW = 1024    # the window the autotuner picks for this batch (bench.py --workload ship256-d5-batch)


def batch_subset_leg(opmos, torch, stream, world: int, rank: int, steps: int) -> dict:
    """Batched form against one query per launch on the SAME queries: a fixed
    subset of the 5-objective ship-grid batch (config 4), run as one
    continuous-batching launch and as a loop of single-query launches, with
    the batch kernel's roofline (algorithmic bytes of the launch over its
    device time). Under torchrun each rank takes its share of the subset."""
    g, q = synth.config4(1)
    sub = q[::BATCH_EVERY]
    mine = shard_queries(len(sub), rank, world, grid_distance(g, sub))
    qs = [sub[i] for i in mine]
    G = opmos.opmos_graph.from_synth(g)
    starts, goals = [s for s, _ in qs], [t for _, t in qs]
    bopt = opmos._options(stream=stream.cuda_stream, window=BATCH_WINDOW, flags=opmos.FLAG_GRAPH)
    sopt = opmos.opmos_default_options(stream=stream.cuda_stream)
    opmos.opmos_solve_batch(G, starts, goals, options=bopt)  # warm-up
    torch.cuda.synchronize()
    times, out = [], None
    for _ in range(max(1, steps)):
        barrier()
        t0 = time.perf_counter()
        out = opmos.opmos_solve_batch(G, starts, goals, options=bopt)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    bsec = max_over_ranks(statistics.median(times))
    barrier()
    t0 = time.perf_counter()
    singles = [opmos.opmos_solve(G, s, t, options=sopt) for s, t in qs]
    torch.cuda.synchronize()
    ssec = max_over_ranks(time.perf_counter() - t0)
    ok = sum(1 for st, r in out if st == opmos.OK)
    same = all(st == opmos.OK and np.array_equal(r.costs, x.costs) for (st, r), x in zip(out, singles))
    rs = [r for _, r in out if r is not None]
    launches = {}
    for r in rs:  # queries re-run in a later launch carry that launch's time
        launches.setdefault(r.stats["search_ns"], []).append(r.stats["bytes"])
    kern_ns = max(launches, key=lambda k: len(launches[k]))
    kbytes = sum(launches[kern_ns])
    peak, src = _peak()
    ach = kbytes / (kern_ns / 1e9) / 1e9
    nq = len(sub)
    return {"workload": f"ship256-d5-batch subset: {nq} of the 1,024 config-4 queries (every {BATCH_EVERY}th), "
                        f"5 objectives, seed 1, window {BATCH_WINDOW}",
            "queries": nq, "queries_ok": ok, "same_fronts_as_single": same,
            "batched_qps": nq / bsec, "one_query_per_launch_qps": nq / ssec,
            "batched_over_single": ssec / bsec, "batch_wall_ms": 1e3 * bsec, "single_loop_ms": 1e3 * ssec,
            "batch_kernel_ms": kern_ns / 1e6,
            "labels_per_s": sum(r.stats["extracted"] for r in rs) / (kern_ns / 1e9),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "kernel": f"multi_kernel<5>", "peak_source": src,
                         "bytes": kbytes, "queries_in_launch": len(launches[kern_ns])}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    g, q = synth.config2()
    s, t = q[0]
    for _ in range(args.warmup):
        cpu_sample(g, s, t, args.cpu_labels)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(g, s, t, args.cpu_labels))
    wall = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config():
    return {"workload": "ship256-d3: 256x256 8-connected ship grid, 3 objectives (length, length x current, "
                        "length x wave), 5% land, corner to corner, seed 1",
            "queries_per_step": 1, "nodes": 65536, "objectives": 3,
            "l2": "flushed: a 256 MiB buffer (larger than L2) is written before every timed step; within a "
                  "step the hot frontier and P entries stay in L2 (88% hit rate measured)"}


def _peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def run_small(args, opmos, torch, stream):
    """128x128 ship grid, one query: the small case for profiler captures."""
    g, q = synth.ship_grid(2, 128, 3)
    s, t = q[0]
    G = opmos.opmos_graph.from_synth(g)
    opt = opmos.opmos_default_options(stream=stream.cuda_stream, window=args.window or None)
    for _ in range(args.warmup):
        opmos.opmos_solve(G, s, t, options=opt)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        r = opmos.opmos_solve(G, s, t, options=opt)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    st = r.stats
    peak, src = _peak()
    ach = st["bytes"] / (st["search_ns"] / 1e9) / 1e9
    print(json.dumps({"metric": "labels/s (GPU extractions, small profiling case)", "value": st["extracted"] / (ms / 1e3),
                      "unit": "labels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
                      "config": {"workload": "ship128-d3: 128x128 ship grid, d=3, corner to corner, seed 2"},
                      "front_size": int(r.costs.shape[0]), "search_kernel_ms": st["search_ns"] / 1e6,
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                   "frac": ach / peak, "peak_source": src}}), flush=True)


def run_batch(args, opmos, torch, stream):
    """Config 4: 1,024 queries in one continuous-batching launch."""
    world, rank, _ = dist_setup()
    g, q = synth.config4(1)
    G = opmos.opmos_graph.from_synth(g)
    mine = shard_queries(len(q), rank, world, grid_distance(g, q))
    starts = [q[i][0] for i in mine]
    goals = [q[i][1] for i in mine]
    # autotuned on a calibration subset (every 32nd query), outside the timed region
    from paper_2411_16667_gb300 import autotune
    calib = q[::32]
    ch = autotune.autotune(G, calib, mode="batch", windows=(128, 256, 1024), lanes=(8, 16), tiles=(32, 64),
                           stream_ptr=stream.cuda_stream)
    # the window of the queries that outgrow the shared launch (alone_labels):
    # tuned on the calibration queries farthest apart, solved alone
    dist = grid_distance(g, calib)
    far = [calib[i] for i in sorted(range(len(calib)), key=lambda i: -dist[i])[:4]]
    alone_window = autotune.autotune(G, far, mode="single", windows=(1024, 4096, 16384, 65536), lanes=(8,),
                                     tiles=(32,), stream_ptr=stream.cuda_stream).window
    opt = ch.options(stream=stream.cuda_stream, flags=opmos.FLAG_GRAPH, alone_window=alone_window)
    if args.window:
        opt.window = args.window
    for _ in range(args.warmup):
        opmos.opmos_solve_batch(G, starts, goals, options=opt)
    torch.cuda.synchronize()
    times, stats = [], None
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            barrier()
            t0 = time.perf_counter()
            out = opmos.opmos_solve_batch(G, starts, goals, options=opt)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    ok = sum(1 for st, _ in out if st == opmos.OK)
    rs = [r for _, r in out if r is not None]
    sec = max_over_ranks(statistics.median(times))
    if rank != 0:
        return
    # one query per launch on an evenly spaced sample of the same queries,
    # with the window the batch gives the queries it solves alone
    sample = q[::16]
    single = opmos.opmos_default_options(stream=stream.cuda_stream, window=alone_window)
    t0 = time.perf_counter()
    for s_, t_ in sample:
        opmos.opmos_solve(G, s_, t_, options=single)
    torch.cuda.synchronize()
    single_qps = len(sample) / (time.perf_counter() - t0)
    cpu = None if args.no_cpu_baseline else cpu_batch_sample(g, q, 32, 2_000_000)
    print(json.dumps({"metric": "batched queries/s", "value": len(q) / sec, "unit": "queries/s", "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
                      "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
                      "data": "synthetic", "cpu_baseline": cpu,
                      "config": {"workload": "ship256-d5-batch: 1,024 queries, Chebyshev 16-128, 5 objectives, seed 1",
                                 "parallelism": f"queries split round-robin over {world} GPU(s)"},
                      "queries_ok": ok, "labels_extracted": sum(r.stats["extracted"] for r in rs),
                      "labels_per_s": sum(r.stats["extracted"] for r in rs) / sec,
                      "batch_kernel_ms": statistics.median(r.stats["search_ns"] for r in rs) / 1e6,
                      "queries_alone": sum(1 for r in rs if r.stats["search_ns"] != statistics.median_low(
                          x.stats["search_ns"] for x in rs)),
                      "alone_labels": opt.alone_labels or 1_000_000, "alone_window": alone_window,
                      "heuristic_ms": rs[0].stats["heuristic_ns"] / 1e6,
                      "one_query_per_launch_qps": single_qps,
                      "one_query_per_launch_sample": f"{len(sample)} of the 1,024 queries (every 16th)",
                      "batched_over_single": (len(q) / sec) / single_qps,
                      "autotuned": {"window": ch.window, "lanes_per_label": ch.lanes_per_label, "tile": ch.tile,
                                    "calibration": f"{len(calib)} queries (every 32nd)", "trials": len(ch.table)},
                      "launch": "one cooperative persistent kernel per batch, captured in a CUDA graph",
                      "clocks": clk.summary()}), flush=True)


def query_hops(g, queries) -> list[int]:
    """Hop distance of each (start, goal) (breadth-first, on the host): used
    to pick the road-graph queries an exact search can finish."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    a = sp.csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.rowptr.astype(np.int64)), shape=(g.n, g.n))
    out = []
    for lo in range(0, len(queries), 32):
        part = queries[lo:lo + 32]
        dist = shortest_path(a, unweighted=True, indices=[s for s, _ in part])
        out += [int(dist[j, t]) for j, (_, t) in enumerate(part)]
    return out


def run_road_batch(args, opmos, torch, stream):
    """Config 3 at its full d = 4: the K queries with the fewest hops among
    the 256 (the ones an exact search can finish: the two i.i.d. random
    objectives make fronts of tens of thousands of vectors), in one
    persistent launch, each under a label budget (Sec. 6.1 reports runs past
    a time limit as timed out; a label budget is the deterministic form of
    that limit), against one query per launch on the same queries. value =
    exact fronts delivered per second; over-budget answers are counted
    apart."""
    world, rank, _ = dist_setup()
    g, q = synth.config3()
    hops = query_hops(g, q)
    sel = sorted(sorted(range(len(q)), key=lambda i: (hops[i], i))[:args.road_queries])
    qs = [q[i] for i in sel]
    G = opmos.opmos_graph.from_synth(g)
    budget = args.road_label_budget
    w = args.window or 1024  # the same window for both arms
    opt = opmos._options(stream=stream.cuda_stream, flags=opmos.FLAG_GRAPH, label_budget=budget, window=w)
    mine = shard_queries(len(qs), rank, world, [hops[i] for i in sel])
    starts = [qs[i][0] for i in mine]
    goals = [qs[i][1] for i in mine]
    for _ in range(args.warmup):
        opmos.opmos_solve_batch(G, starts, goals, options=opt)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            barrier()
            t0 = time.perf_counter()
            out = opmos.opmos_solve_batch(G, starts, goals, options=opt)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
    sec = max_over_ranks(statistics.median(times))
    single = opmos._options(stream=stream.cuda_stream, label_budget=budget, flags=opmos.FLAG_NO_PATHS, window=w)
    barrier()
    t0 = time.perf_counter()
    sstat = []
    for s_, t_ in zip(starts, goals):
        try:
            opmos.opmos_solve(G, s_, t_, options=single)
            sstat.append(opmos.OK)
        except opmos.OpmosError as e:
            if e.code != opmos.ERR_BUDGET:
                raise
            sstat.append(e.code)
    torch.cuda.synchronize()
    ssec = max_over_ranks(time.perf_counter() - t0)
    if rank != 0:
        return
    ok = sum(1 for st, _ in out if st == opmos.OK)
    over = sum(1 for st, _ in out if st == opmos.ERR_BUDGET)
    rs = [r for _, r in out if r is not None]
    print(json.dumps({"metric": "batched queries/s (exact fronts)", "value": world * ok / sec, "unit": "queries/s",
                      "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
                      "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
                      "data": "synthetic",
                      "config": {"workload": f"road200k-d4-batch: the {len(qs)} fewest-hop of the 256 queries "
                                             f"(hops {min(hops[i] for i in sel)}-{max(hops[i] for i in sel)}), "
                                             f"4 objectives, seed 1, label budget {budget} per query, window {w}",
                                 "parallelism": f"queries split over {world} GPU(s) by hop count"},
                      "queries": len(qs), "queries_ok": ok, "queries_over_budget": over,
                      "answered_per_s": world * len(starts) / sec,
                      "front_sizes": sorted(int(r.costs.shape[0]) for r in rs),
                      "labels_extracted_ok": sum(r.stats["extracted"] for r in rs),
                      "one_query_per_launch_ok_per_s": world * sstat.count(opmos.OK) / ssec,
                      "one_query_per_launch_ms": 1e3 * ssec,
                      "batched_over_single": ssec / sec,
                      "launch": "one cooperative persistent kernel per batch, captured in a CUDA graph",
                      "clocks": clk.summary()}), flush=True)


def run_order(args, opmos, torch, stream):
    """Ordered (lexicographic priority) windows against FIFO windows (Sec. 4
    and 7.1: PQ versus FIFO) at the same width: work (labels extracted, work
    ratio against the oracle) and time on the config-2 query, the d = 12
    route, and the config-4 batch subset."""
    fx = fixture_stats()
    g, q = synth.config2()
    G = opmos.opmos_graph.from_synth(g)
    rows = []
    for w in (256, 1024, 4096, 16384, 65536, 262144):
        for name, flags in (("ordered", 0), ("fifo", opmos.FLAG_FIFO)):
            opt = opmos.opmos_default_options(stream=stream.cuda_stream, window=w, flags=flags)
            r = opmos.opmos_solve(G, *q[0], options=opt)
            ok = r.costs.shape[0] == fx["count"]
            rows.append({"workload": "ship256-d3", "order": name, "window": w, "front_ok": ok,
                         "search_ms": r.stats["search_ns"] / 1e6, "steps": r.stats["steps"],
                         "extracted": r.stats["extracted"], "work_ratio": r.stats["extracted"] / fx["extracted"]})
            print(json.dumps(rows[-1]), flush=True)
    for w in (256, 1024):
        for name, flags in (("ordered", 0), ("fifo", opmos.FLAG_FIFO)):
            leg = route_leg(opmos, torch, stream, 1, window=w, flags=flags)
            rows.append({"workload": "route6x8x24-d12", "order": name, "window": w,
                         "front_ok": leg["front_matches_oracle"], "search_ms": leg["search_kernel_ms"],
                         "steps": leg["steps"], "extracted": leg["gpu_labels_extracted"],
                         "work_ratio": leg["work_ratio"]})
            print(json.dumps(rows[-1]), flush=True)
    g4, q4 = synth.config4(1)
    G4 = opmos.opmos_graph.from_synth(g4)
    sub = q4[::BATCH_EVERY]
    for name, flags in (("ordered", 0), ("fifo", opmos.FLAG_FIFO)):
        opt = opmos._options(stream=stream.cuda_stream, window=BATCH_WINDOW, flags=flags)
        out = opmos.opmos_solve_batch(G4, [s for s, _ in sub], [t for _, t in sub], options=opt)
        rs = [r for _, r in out if r is not None]
        rows.append({"workload": f"ship256-d5-batch subset ({len(sub)} queries)", "order": name,
                     "window": BATCH_WINDOW, "queries_ok": sum(1 for st_, _ in out if st_ == opmos.OK),
                     "batch_kernel_ms": max(r.stats["search_ns"] for r in rs) / 1e6,
                     "extracted": sum(r.stats["extracted"] for r in rs)})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": "work and time, ordered vs FIFO windows", "rows": len(rows)}), flush=True)


def serve_queries(n, seed=5):
    """Config-5 query stream over configs 1-3: graph uniform, d ~ U{2..5}
    clamped to the graph's objective count, start/goal as in each config."""
    g1, q1 = synth.config1()
    g2, q2 = synth.config2()
    g3, q3 = synth.config3()
    graphs = [g1, g2, g3]
    qsets = [q1, q2, q3]
    out = []
    for i in range(n):
        gi = int(synth.rand_int(seed, 900, i, 0, 2))
        d = min(int(synth.rand_int(seed, 901, i, 2, 5)), graphs[gi].d)
        qs = qsets[gi]
        s, t = qs[int(synth.rand_int(seed, 902, i, 0, len(qs) - 1))]
        out.append((gi, d, s, t))
    return graphs, out


def run_serve(args, opmos, torch, stream):
    """Config 5: continuous-batching server under Poisson arrivals."""
    import random
    budget = args.serve_label_budget
    n = args.serve_queries
    graphs, plan = serve_queries(n)
    G = [opmos.opmos_graph.from_synth(g) for g in graphs]
    # one query per launch over the same query list (no server resident)
    single = opmos.opmos_default_options(stream=stream.cuda_stream, label_budget=budget, window=args.window or 256)
    t0 = time.perf_counter()
    n_single = n
    single_status = []
    for gi, d, s, t in plan:
        single.d_used = d
        try:
            opmos.opmos_solve(G[gi], s, t, options=single)
            single_status.append(0)
        except opmos.OpmosError as e:
            single_status.append(e.code)
    torch.cuda.synchronize()
    single_qps = n_single / (time.perf_counter() - t0)
    srv = opmos.opmos_server(G, label_budget=budget, window=args.window or 256)

    def run(queries, rate):
        """Submit with Poisson arrivals at `rate` q/s (0: all at once)."""
        rnd = random.Random(7)
        pending, lat, status = {}, [], []
        t_next = time.perf_counter()
        i = 0
        t_start = time.perf_counter()
        while i < len(queries) or pending:
            now = time.perf_counter()
            while i < len(queries) and now >= t_next:
                try:
                    tk = srv.submit(*queries[i])
                    pending[tk] = time.perf_counter()
                    i += 1
                    t_next += rnd.expovariate(rate) if rate > 0 else 0.0
                except opmos.OpmosError:
                    break  # queue full: retry on the next pass
                now = time.perf_counter()
            for tk in list(pending):
                st, _ = srv.poll(tk)
                if st != opmos.PENDING:
                    lat.append(time.perf_counter() - pending.pop(tk))
                    status.append(st)
            time.sleep(0.0005)
        wall = time.perf_counter() - t_start
        lat.sort()
        return {"queries": len(queries), "qps": len(queries) / wall,
                "p50_ms": 1e3 * lat[len(lat) // 2], "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "ok": sum(1 for x in status if x == opmos.OK),
                "budget_exceeded": sum(1 for x in status if x == opmos.ERR_BUDGET),
                "capacity": sum(1 for x in status if x == opmos.ERR_CAPACITY)}

    sat = run(plan, 0.0)
    rates = {}
    with ClockSampler(0) as clk:
        for frac in (0.25, 0.5, 0.9):
            r = frac * sat["qps"]
            rates[f"{frac:.2f}x"] = {"rate_qps": r, **run(plan, r)}
    srv.close()
    best = max(v["qps"] for v in rates.values())
    print(json.dumps({"metric": "served queries/s and p50/p99 latency", "value": sat["qps"], "unit": "queries/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
                      "config": {"workload": "serve: configs 1-3 graphs resident, d ~ U{2..5} clamped, Poisson arrivals;"
                                             " the same query list at saturation, at each rate and one query per launch",
                                 "label_budget_per_query": budget, "queries_per_rate": n},
                      "saturation": sat, "rates": rates, "one_query_per_launch_qps": single_qps,
                      "one_query_per_launch_ok": sum(1 for x in single_status if x == 0),
                      "one_query_per_launch_over_budget": sum(1 for x in single_status if x == opmos.ERR_BUDGET),
                      "served_over_single": sat["qps"] / single_qps, "best_rate_qps": best,
                      "clocks": clk.summary()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="opmos", choices=["opmos", "reference"])
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--cpu-labels", type=int, default=CPU_SAMPLE_LABELS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch-leg", action="store_true",
                    help="leave the config-4 batch subset out of the default line")
    ap.add_argument("--serve-queries", type=int, default=300)
    ap.add_argument("--serve-label-budget", type=int, default=1_000_000)
    ap.add_argument("--road-label-budget", type=int, default=5_000_000)
    ap.add_argument("--road-queries", type=int, default=32)
    ap.add_argument("--workload", default="ship256-d3",
                    choices=["ship256-d3", "ship128-d3", "ship256-d5-batch", "road200k-d4-batch", "serve",
                             "order"])
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload != "ship256-d3":
        stream = torch.cuda.Stream()
        try:
            with torch.cuda.stream(stream):
                if args.workload == "ship128-d3":
                    return run_small(args, opmos, torch, stream)
                if args.workload == "ship256-d5-batch":
                    return run_batch(args, opmos, torch, stream)
                if args.workload == "road200k-d4-batch":
                    return run_road_batch(args, opmos, torch, stream)
                if args.workload == "order":
                    return run_order(args, opmos, torch, stream)
                return run_serve(args, opmos, torch, stream)
        finally:
            if world > 1:
                torch.distributed.destroy_process_group()
    stream = torch.cuda.Stream()
    g, q = synth.config2()
    s, t = q[0]
    fx = fixture_stats()
    if g.digest() != fx["digest"]:
        raise RuntimeError("regenerated workload does not match the oracle fixture")
    useful = fx["extracted"]
    # the window: autotuned on the same recipe's grid of the next seed (outside
    # the timed region), unless --window is given
    window = args.window or tuned_window(opmos, stream, *synth.ship_grid(2, 256, 3),
                                         (1024, 4096, 16384, 65536, 262144))
    G = opmos.opmos_graph.from_synth(g)
    opt = opmos.opmos_default_options(stream=stream.cuda_stream, window=window)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        return opmos.opmos_solve(G, s, t, options=opt)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            res = step()
        if res.costs.shape[0] != fx["count"]:
            raise RuntimeError(f"front size {res.costs.shape[0]} != oracle {fx['count']}")
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stats = []
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                r = step()
                ev[i][1].record(stream)
                stats.append(r.stats)
            torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        ms = sum(step_ms) / len(step_ms)
        ms = max_over_ranks(ms)

        # end to end through the C ABI with host buffers
        h2d = g.rowptr.nbytes + g.col.nbytes + g.cost.nbytes
        e2e_t, d2h = [], 0
        for i in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Gh = opmos.opmos_graph.from_synth(g)
            r = opmos.opmos_solve(Gh, s, t, options=opt)
            Gh.close()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
            d2h = r.costs.nbytes + sum(a.nbytes // 2 + b.nbytes for a, b in r.paths)  # device words are u32

        batch = None if args.no_batch_leg else batch_subset_leg(opmos, torch, stream, world, rank, 1)
        route = None if args.no_batch_leg else route_leg(opmos, torch, stream, 3)

    search_ns = statistics.median(x["search_ns"] for x in stats)
    heur_ns = statistics.median(x["heuristic_ns"] for x in stats)
    st = stats[-1]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    achieved = st["bytes"] / (search_ns / 1e9) / 1e9
    achieved_oc = oracle_count_bytes(fx, g.d) / (search_ns / 1e9) / 1e9
    launch = (opt.window, opt.lanes_per_label, opt.tile, opt.delta)
    traffic = TRAFFIC.get(kernel_source_digest(launch))
    value = world * useful / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": workload_config(),
        "time_to_front_ms": ms, "heuristic_ms": heur_ns / 1e6, "search_kernel_ms": search_ns / 1e6,
        "gpu_labels_extracted": st["extracted"], "oracle_labels_extracted": useful,
        "work_ratio": st["extracted"] / useful, "gpu_labels_per_s": st["extracted"] / (ms / 1e3),
        "candidates_per_s": st["candidates"] / (ms / 1e3), "front_size": int(fx["count"]),
        "search_steps": st["steps"], "step_ms_all": step_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "search_grid_kernel",
                     "achieved_oracle_count": achieved_oc, "frac_oracle_count": achieved_oc / peak,
                     "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                     else "fallback 6.8 TB/s"},
        "e2e": {"value": world * useful / statistics.median(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
        "open_scanned_per_step": st["open_scanned"] / max(1, st["steps"]),
        "longest_task_us_per_step": {k: v / 1e3 / max(1, st["steps"]) for k, v in
                                     zip(("block_merge", "warp_merge", "extraction"), st["longest_task_ns"])},
        "window": opt.window,
        "window_choice": "autotuned on the 256x256 ship grid of seed 2 (same recipe, corner query): the fastest "
                         "of 1024 ... 262144" if not args.window else "given",
    }
    if batch is not None:
        line["batch"] = batch
    if route is not None:
        line["route_d12"] = route
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample(g, s, t, args.cpu_labels)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
