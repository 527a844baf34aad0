"""Benchmark: Tabu moves evaluated per second on the large single instance.

Workload (one "step"): one complete Tabu search of 10,000 iterations on the large
instance (40 bases, 50 vehicles, 200 clustered facilities in a 3000 km box, 400
Zipf-skewed missions, tenure 15, duty cap 960 min as a penalty with lambda 1000), greedy
start included, through asched_tabu_solve on its planned launch shape (every thread-block
cluster the device holds at once). Every iteration evaluates all M(M+V-2) + M(M-1)/2 =
259,000 moves, so a step is 2.59 G moves. The paper-shaped instance (100 missions, 5,000
iterations) is reported beside it, then the batched, serving, sweep and travel-matrix
workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own copy of the single instances (a single search
does not shard): the line reports the sum of all ranks' moves over the slowest rank's
time. Batches and request streams are sharded: each rank takes its own part of the
1,024 instances (a contiguous block) and of the request stream (every N-th request).
`--impl reference` times the plain CPU oracle on this host's cores instead (bounded
iteration samples of the same instance).
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Tabu moves evaluated/sec (bit-exact); batched solves/sec and p50/p99 latency"
UNIT = "moves/s"
WORKLOADS = {
    "large": ("large single instance: 40 bases, 50 vehicles, 200 facilities in 4 Gaussian clusters "
              "(sigma 80 km) + 20% uniform outliers in a 3000 km box, 400 missions Zipf(1.1) over "
              "facilities, int32 minutes at 250 km/h, duty cap 960 min (penalty, lambda 1000), "
              "tenure 15, 10,000 iterations, greedy start"),
    "paper_shaped": ("paper-shaped single instance: 12 bases, 20 vehicles, 60 facilities in 4 Gaussian "
                     "clusters (sigma 80 km) + 20% uniform outliers in a 1500 km box, 100 uniform "
                     "missions, int32 minutes at 250 km/h, duty cap 720 min (penalty, lambda 1000), "
                     "tenure 10, 5,000 iterations, greedy start"),
}
# Algorithmic work per evaluated move, counted from the formulas of the hot path
# (removal + insertion cost, penalty of the touched routes, compatibility, tabu,
# aspiration, admissibility, key): a relocation is about 20 int32 operations and 3
# shared-memory gathers (two travel-table entries and one tabu stamp); a swap about 30
# operations and 6 gathers (four table entries, two stamps).
OPS_RELOCATE, OPS_SWAP = 20, 30
GATHERS_RELOCATE, GATHERS_SWAP = 3, 6
# DRAM bytes (read + write) per launch of the headline kernel from one ncu capture,
# keyed by the first 16 hex digits of the SHA-256 of csrc/asched.cu it was taken on;
# any other source reports traffic as null.
TRAFFIC_BYTES = {"047155f641486d20": 916224}  # ncu launch list of the large-instance bench, mean of 12 launches


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


TIMING_BACK_TO_BACK = "device time per call: 5 calls back to back between CUDA events, median of 3 such runs"


def device_ms(fn, reps=5, rounds=3):
    """Device time per call of fn (which queues work on the current stream): reps calls
    back to back between two CUDA events, so the host queues ahead and its own time per
    call (argument checks, Python) does not leave the device idle; median over rounds."""
    import torch

    ts = []
    for _ in range(rounds):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / reps)
    return statistics.median(ts)


def source_sha():
    src = os.path.join(ROOT, "paper_2002_11710_gb300", "csrc", "asched.cu")
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def moves_split(M, V):
    return M * (M + V - 2), M * (M - 1) // 2


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(name):
    from paper_2002_11710_gb300 import gen

    if name == "large":
        return gen.large(0), gen.LARGE_PARAMS
    return gen.paper_shaped(0), gen.PAPER_SHAPED_PARAMS


def cpu_oracle_sample(inst, p, iterations, threads):
    """The oracle as it stands on the first `iterations` iterations, its loop over moves
    on `threads` OpenMP threads (0: every core). Returns (moves/s, seconds, threads)."""
    import oracle

    used = oracle.set_threads(threads)
    pb = oracle.Problem(inst, p.cap_mode, p.lam)
    t0 = time.perf_counter()
    r = oracle.tabu_search(pb, p.tenure, iterations)
    dt = time.perf_counter() - t0
    assert r["status"] == 0
    M, V = inst.n_missions, inst.n_vehicles
    n = (M * (M + V - 2) + M * (M - 1) // 2) * iterations
    return n / dt, dt, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def max_over_ranks(seconds, world, device):
    """The slowest rank's time (all ranks call this; world 1 returns the input)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_arrays(a, world):
    """Every rank's numpy array concatenated (all ranks call this)."""
    if world <= 1:
        return a
    import torch.distributed as dist

    parts = [None] * world
    dist.all_gather_object(parts, np.asarray(a))
    return np.concatenate(parts)


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args, rank, world):
    """The reference arm: the oracle on the headline workload, on every host core,
    each step the first --ref-iterations iterations."""
    if rank != 0:
        return
    inst, p = workload("large")
    it_sample = args.ref_iterations
    threads = 0
    for _ in range(args.warmup):
        cpu_oracle_sample(inst, p, it_sample, threads)
    rates, times, used = [], [], 1
    for _ in range(args.steps):
        r, dt, used = cpu_oracle_sample(inst, p, it_sample, threads)
        rates.append(r)
        times.append(dt)
    M, V = inst.n_missions, inst.n_vehicles
    n = (M * (M + V - 2) + M * (M - 1) // 2) * it_sample
    value = n * len(times) / sum(times)
    sample = (f"first {it_sample} of 10,000 iterations of the large instance per step, "
              f"oracle's loop over moves on {used} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["large"], "sample": sample, "n_missions": M, "n_vehicles": V},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_single(name, args, dev, world, flush, barrier, clocks=None):
    """One single-instance workload: warm-up, then `steps` full searches each between
    CUDA events on the launching stream (L2 flushed before each, untimed), then the same
    searches end to end from pinned host buffers."""
    import torch

    from paper_2002_11710_gb300 import api

    inst, p = workload(name)
    if args.iterations > 0:  # a shorter search of the same instance (profiling)
        p = dataclasses.replace(p, iterations=args.iterations)
    M, V = inst.n_missions, inst.n_vehicles
    R, S = moves_split(M, V)
    params = api.params_from(p, cluster_size=args.cluster, block_threads=args.threads, grid_clusters=args.grid,
                             plain_launch=args.plain_launch)
    dp = api.DeviceProblem(inst, dev)
    plan = api.plan(dp, params)
    out = api.alloc_output(dp, p.iterations)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        api.solve(dp, params, out=out)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    if info[api.INFO_STATUS] != 0:
        raise RuntimeError(f"{name}: device status {info[api.INFO_STATUS]}")
    z_best = int(info[api.INFO_Z_BEST])
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)  # evict the previous step's data from L2 (not timed)
        starts[k].record(stream)
        api.solve(dp, params, out=out)
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = max_over_ranks(sum(step_ms) / 1000.0, world, dev)
    # end to end through the public API from pinned host data
    pinned = api.pin_instance(inst)
    e2e_times = []
    h2d, d2h = pinned.nbytes(), 0
    for k in range(args.warmup + args.steps):
        barrier()
        flush.fill_(k)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        res = api.solve_host(pinned, params, device=dev)
        t2 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t2 - t1)
        d2h = sum(int(v.nbytes) for v in res.values())
        assert int(res["info"][api.INFO_Z_BEST]) == z_best
    e2e_s = max_over_ranks(sum(e2e_times), world, dev)
    moves_step = (R + S) * p.iterations
    return {"inst": inst, "p": p, "plan": plan, "R": R, "S": S, "step_ms": step_ms, "dev_s": dev_s,
            "e2e_s": e2e_s, "wall": wall, "clocks": clk, "z_best": z_best, "moves_step": moves_step,
            "h2d": h2d, "d2h": d2h,
            "value": whole_job_rate(moves_step * args.steps, world, dev_s),
            "e2e_value": whole_job_rate(moves_step * args.steps, world, e2e_s)}


# One warp instruction per clock from each of an SM's four schedulers: 128 int32 lanes
# per clock per SM is the issue bound of any integer instruction mix.
ISSUE_LANES_PER_CLK_SM = 128


def roofline(r, peaks, sms, sm_max_mhz, traffic):
    """The hot kernel's roofline: algorithmic int32 operations and shared-memory gathers
    per launch over its mean launch time, against the chip's integer issue rate at its
    maximum SM clock: the larger of the issue bound (128 lanes per clock per SM) and the
    best rate the int32 probes measured (add / xor / min and add / xor mixes)."""
    launch_s = statistics.mean(r["step_ms"]) / 1000.0
    its = r["p"].iterations
    ops = (r["R"] * OPS_RELOCATE + r["S"] * OPS_SWAP) * its
    gathers = (r["R"] * GATHERS_RELOCATE + r["S"] * GATHERS_SWAP) * its
    clk = sm_max_mhz * 1e6
    measured = max(peaks["int32_ops_per_clk_sm"], peaks.get("int32_add_xor_ops_per_clk_sm", 0.0))
    per_clk = max(ISSUE_LANES_PER_CLK_SM, measured)
    peak_ops = per_clk * sms * clk / 1e12
    achieved = ops / launch_s / 1e12
    used = r["plan"].cluster_size * r["plan"].grid_clusters
    g_rate = gathers / launch_s
    basis = (f"max(issue bound {ISSUE_LANES_PER_CLK_SM} int32 lanes/clk/SM, best measured int32 mix "
             f"{measured:.1f} ops/clk/SM) x {sms} SMs x {sm_max_mhz:.0f} MHz")
    return {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s", "frac": achieved / peak_ops,
            "traffic": traffic,
            "peak_basis": basis,
            "ops_per_move": {"relocate": OPS_RELOCATE, "swap": OPS_SWAP},
            "sms_used": used, "frac_of_sms_used": achieved / (peak_ops * used / sms),
            "smem": {"gathers_per_s": g_rate,
                     "frac_of_gather_peak": g_rate / (peaks["lds_gather_words_per_clk_sm"] * sms * clk),
                     "frac_of_conflict_free_peak": g_rate / (peaks["lds_words_per_clk_sm"] * sms * clk),
                     "gathers_per_move": {"relocate": GATHERS_RELOCATE, "swap": GATHERS_SWAP}}}


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2002_11710_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = Clocks(local_rank) if rank == 0 else None
    head = time_single("large", args, dev, world, flush, barrier, clocks)
    second = time_single("paper_shaped", args, dev, world, flush, barrier) if args.paper_shaped else None
    peaks_file = read_peaks()
    sm_max_mhz = float(peaks_file.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probes = api.measure_sm_peaks(dev)
    batched = run_batched(args, dev, rank, world) if args.batched else None
    serving = run_serving(args, dev, rank, world) if args.serve_seconds > 0 else None
    sweeps = run_sweeps(args, dev) if args.sweeps else None
    if rank != 0:
        return
    inst, p = head["inst"], head["p"]
    M, V = inst.n_missions, inst.n_vehicles
    traffic = TRAFFIC_BYTES.get(source_sha())
    cpu = None
    if world == 1 and args.cpu_iterations > 0:
        r1, dt1, _ = cpu_oracle_sample(inst, p, args.cpu_iterations, 1)
        rn, dtn, used = cpu_oracle_sample(inst, p, args.cpu_iterations_all, 0)
        cpu = {"value": rn, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": (f"first {args.cpu_iterations_all} of 10,000 iterations of the large instance, "
                          f"{dtn:.1f} s on {used} threads (host has {host_cores()} cores)"),
               "one_core": {"value": r1, "cores": 1,
                            "sample": f"first {args.cpu_iterations} iterations, {dt1:.1f} s"}}
    lat = sorted(head["step_ms"])
    plan = head["plan"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(head["step_ms"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS["large"], "n_missions": M, "n_vehicles": V,
                   "iterations": p.iterations, "moves_per_iteration": head["R"] + head["S"],
                   "moves_per_step": head["moves_step"], "cluster_size": plan.cluster_size,
                   "grid_clusters": plan.grid_clusters, "block_threads": plan.block_threads,
                   "smem_bytes": plan.smem_bytes,
                   "l2": "flushed between steps (256 MB write, untimed)",
                   "parallelism": "one instance per GPU (replicas); batches and streams sharded"},
        "solves_per_s": world * args.steps / head["dev_s"],
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "wall_s": head["wall"],
        "z_best": head["z_best"],
        "gpu_launches": args.steps,
        "e2e": {"value": head["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": head["h2d"],
                "d2h_bytes_per_step": head["d2h"]},
        "roofline": roofline(head, probes, sms, sm_max_mhz, traffic),
        "sm_peaks_measured": probes,
        "paper_shaped": None if second is None else {
            "workload": WORKLOADS["paper_shaped"], "value": second["value"], "unit": UNIT,
            "ms_per_step": statistics.mean(second["step_ms"]),
            "e2e": {"value": second["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": second["h2d"],
                    "d2h_bytes_per_step": second["d2h"]},
            "launch_shape": {"cluster_size": second["plan"].cluster_size,
                             "grid_clusters": second["plan"].grid_clusters,
                             "block_threads": second["plan"].block_threads},
            "roofline": roofline(second, probes, sms, sm_max_mhz, None), "z_best": second["z_best"]},
        "batched": batched,
        "serving": serving,
        "sweeps": sweeps,
        "cpu_baseline": cpu,
        "clocks": head["clocks"],
    }
    print(json.dumps(line), flush=True)


def _shape_name(c):
    """'threads[/int16][/xC]' for an autotune candidate (threads, compact, CTAs per instance)."""
    return f"{c[0]}{'/int16' if c[1] else ''}{f'/x{c[2]}' if c[2] > 1 else ''}"


def run_batched(args, dev, rank, world):
    """The batched workload: 1,024 instances (V ~ U[3, 30], M ~ U[10, 200], paper-shaped
    geography, 2,000 iterations each) in one persistent launch replayed from a CUDA graph,
    launch shape picked by the autotuner, against the same instances as single-instance
    launches. Under N ranks each rank solves a contiguous block of the instances."""
    import torch

    from paper_2002_11710_gb300 import api, gen, shard

    lo, hi = shard.contiguous(1024, rank, world)
    insts = [gen.batched_member(i) for i in range(lo, hi)]
    p = gen.BATCHED_PARAMS
    moves = sum(api.num_moves(i.n_missions, i.n_vehicles) for i in insts) * p.iterations
    bp = api.BatchProblem(insts, dev)
    choice, tune = api.autotune_batch(bp, api.params_from(p))
    params = api.tuned_params(api.params_from(p), choice)
    thr = {"block_threads": choice[0], "layout": "int16 matrix" if choice[1] else "gather tables",
           "ctas_per_instance": choice[2], "moves_per_warp": api.batch_moves_per_warp(bp, choice)}
    graph, out = api.capture_batch(bp, params)
    for _ in range(max(1, args.warmup // 2)):
        graph.replay()
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ok = int((out.info.view(-1, api.INFO_LEN)[:, api.INFO_STATUS] == 0).sum())
    single = api.params_from(p)
    dps = [api.DeviceProblem(i, dev) for i in insts]
    outs = [api.alloc_output(d, p.iterations) for d in dps]
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for d, o in zip(dps, outs):
        api.solve(d, single, out=o)
    b.record()
    b.synchronize()
    seq_ms = max_over_ranks(a.elapsed_time(b), world, dev)
    t = max_over_ranks(statistics.median(ms), world, dev)
    moves = sum_over_ranks(moves, world, dev)
    ok = int(sum_over_ranks(ok, world, dev))
    return {"workload": "1,024 instances, V ~ U[3,30], M ~ U[10,200], 2,000 iterations each, "
                        "replayed from a captured CUDA graph",
            "ms": t, "solves_per_s": 1024 / t * 1e3, "moves_per_s": moves / t * 1e3,
            "launch_shape": thr,
            "autotune_ms": {_shape_name(c): v for c, v in tune.items()},
            "autotune_moves_per_warp": {_shape_name(c): api.batch_moves_per_warp(bp, c) for c in tune},
            "instances_ok": ok, "shard": f"contiguous block of {hi - lo} instances per rank ({world} ranks)",
            "sequential_ms": seq_ms, "sequential_solves_per_s": 1024 / seq_ms * 1e3,
            "speedup_vs_sequential": seq_ms / t, "gpu_launches": 2}


# Requests of at least BIG_MISSIONS missions go to a launch of BIG_CLUSTERS clusters of
# BIG_CLUSTER CTAs (chosen by a sweep on this stream: p99 27.1 ms with one-CTA workers
# only, 5.0 ms with this lane).
BIG_MISSIONS, BIG_CLUSTER, BIG_CLUSTERS = 60, 8, 8


def run_plain(reqs, arrivals, params, dev, span_s, max_in_flight=32, max_v=80, max_m=400):
    """The plain per-request path over the stream's span: one asched_tabu_solve launch
    per request in arrival order on one stream, at most max_in_flight queued at once,
    stopped at span_s. Returns (latencies of the served requests, served count, lower
    bounds span_s - arrival for the requests that had arrived but were not served)."""
    import torch

    from paper_2002_11710_gb300 import api

    def z(n):
        return torch.zeros(n, dtype=torch.int32, device=dev)

    ring = 2 * max_in_flight
    outs = [api.SolveOutput(route_off=z(max_v + 1), route=z(max_m), flight=z(max_v), overflow=z(max_v),
                            info=z(api.INFO_LEN), traj_move=None, traj_z=None) for _ in range(ring)]
    evs = [torch.cuda.Event() for _ in range(ring)]
    st = torch.cuda.Stream(device=dev)
    problems = {}
    n = len(reqs)
    lat = []
    pending = collections.deque()
    t0 = time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < span_s:
        while pending and evs[pending[0] % ring].query():
            k = pending.popleft()
            lat.append(time.perf_counter() - t0 - arrivals[k])
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now and len(pending) < max_in_flight:
            dp = problems.get(id(reqs[i]))
            if dp is None:
                dp = problems[id(reqs[i])] = api.DeviceProblem(reqs[i], dev)
            api.solve(dp, params, out=outs[i % ring], stream=st)
            evs[i % ring].record(st)
            pending.append(i)
            i += 1
    st.synchronize()
    arrived = int((arrivals < span_s).sum())
    unserved = [span_s - arrivals[k] for k in range(len(lat), arrived)]
    return np.array(lat), len(lat), np.array(unserved)


def run_serving(args, dev, rank, world):
    """The serving workload: Poisson re-planning requests at 2,000 req/s for
    --serve-seconds (sizes lognormal around 60 missions, clipped to [10, 400],
    V = ceil(M/5), 1,000 iterations each) through the continuous-batching server, with
    slots admitted under a 40 GB device-memory budget; against the plain path (one
    asched_tabu_solve launch per request, in arrival order on one stream) over the same
    span. Under N ranks every rank serves every N-th request of the stream."""
    from paper_2002_11710_gb300 import api, gen, serve, shard

    params = api.params_from(gen.SERVING_PARAMS)
    pool = [gen.serving_request(20_000 + k) for k in range(2048)]
    arrivals_all = gen.poisson_arrivals(7, 2000.0, args.serve_seconds)
    mine = np.array(list(shard.strided(len(arrivals_all), rank, world)), dtype=np.int64)
    arrivals = arrivals_all[mine]
    reqs = [pool[k % len(pool)] for k in mine]
    srv = serve.Server(max_loc=72, max_vehicles=80, max_missions=400, n_slots=4096,
                       budget_bytes=40 << 30, device=dev, big_missions=BIG_MISSIONS,
                       big_cluster=BIG_CLUSTER, big_clusters=BIG_CLUSTERS)
    srv.start(params, idle_timeout_s=60.0)
    try:
        lat, wall = serve.run_stream(srv, reqs, arrivals)
    finally:
        srv.stop()
    served = int(sum_over_ranks(srv.served(), world, dev))
    wall = max_over_ranks(wall, world, dev)
    lat = gather_arrays(lat, world)
    plat, pserved, punserved = run_plain(reqs, arrivals, params, dev, args.serve_seconds)
    pserved = int(sum_over_ranks(pserved, world, dev))
    plat = gather_arrays(plat, world)
    punserved = gather_arrays(punserved, world)
    both = np.concatenate([plat, punserved]) if len(punserved) else plat
    return {"workload": (f"Poisson 2,000 req/s for {args.serve_seconds:g} s, M ~ lognormal(median 60) "
                         "in [10, 400], V = ceil(M/5), 1,000 iterations, 40 GB slot budget"),
            "lanes": {"one_cta": f"requests of fewer than {BIG_MISSIONS} missions, one CTA each",
                      "clusters": f"requests of {BIG_MISSIONS} missions or more, {BIG_CLUSTERS} clusters "
                                  f"of {BIG_CLUSTER} CTAs, one cluster per request"},
            "requests": len(arrivals_all), "served": served, "wall_s": wall,
            "shard": f"every {world}-th request per rank",
            "solves_per_s": len(arrivals_all) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                           "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(lat.max() * 1e3)},
            "slots": srv.n_slots, "slot_bytes": srv.slot_bytes,
            "plain_per_request": {
                "span_s": args.serve_seconds, "served": pserved, "unserved_at_end": int(len(punserved)),
                "solves_per_s": pserved / args.serve_seconds,
                "latency_ms_served": {"p50": float(np.percentile(plat, 50) * 1e3) if len(plat) else None,
                                      "p99": float(np.percentile(plat, 99) * 1e3) if len(plat) else None},
                "latency_ms_all_lower_bound": {"p50": float(np.percentile(both, 50) * 1e3),
                                               "p99": float(np.percentile(both, 99) * 1e3)},
                "note": "requests not served by the end of the span count with latency >= span - arrival"}}


def run_travel_matrix(args, bp, insts, dev):
    """Row f4: every instance's [2][L][L] matrix rebuilt on the device from coordinates
    (asched_travel_matrix) into the batch's travel array, Euclidean on the km coordinates
    and Haversine (Eq. e1) on the same points mapped into a 14 x 21 degree box; checked
    against the host-built matrices (Euclidean: bit for bit). Roofline: the algorithmic
    bytes are the int32 matrix entries written (plus 16 B of coordinates per location)."""
    import torch

    from paper_2002_11710_gb300 import api

    xy = np.concatenate([i.coords for i in insts])
    coords = torch.from_numpy(xy).to(dev, torch.float64)
    ll = torch.from_numpy(np.stack([42.0 + xy[:, 1] / 1000.0 * 14.0, -95.0 + xy[:, 0] / 1000.0 * 21.0],
                                   axis=1)).to(dev, torch.float64)
    want = bp.travel.clone()
    hbm = read_peaks().get("hbm_gbs")
    L = np.diff(bp.h_loc_off).astype(np.int64)
    pairs = int((L * L).sum())
    nbytes = 4 * bp.n_types * pairs + 16 * int(L.sum())
    res = {"workload": f"{bp.B:,} instances, {pairs:,} location pairs, 2 layers (300 / 500 km/h)",
           "bytes_per_launch": nbytes, "gpu_launches": 1, "timing": TIMING_BACK_TO_BACK}
    for name, c, metric in (("euclidean", coords, api.METRIC_EUCLIDEAN), ("haversine", ll, api.METRIC_HAVERSINE)):
        for _ in range(2):
            st = api.travel_into_batch(bp, c, [300.0, 500.0], metric)
        torch.cuda.synchronize()
        t = device_ms(lambda: api.travel_into_batch(bp, c, [300.0, 500.0], metric))
        st = api.travel_into_batch(bp, c, [300.0, 500.0], metric)
        res[name] = {"ms": t, "GB_per_s": nbytes / t / 1e6, "pairs_per_s": pairs / t * 1e3,
                     "status": int(st.item())}
        if hbm:
            res[name]["frac_of_measured_hbm"] = nbytes / t / 1e6 / float(hbm)
        if metric == api.METRIC_EUCLIDEAN:
            res[name]["equals_host_matrices"] = bool(torch.equal(bp.travel, want))
    bp.travel.copy_(want)
    return res


def run_sweeps(args, dev):
    """The paper's own local searches (Algorithm 2, Neighbourhood Search; Algorithm 3 as
    printed, the per-mission sweep) started from Algorithm 1 with its repair, by default on
    65,536 paper-fleet instances (16,384 distinct ones, each four times: 12-33 missions,
    4 plane + 8 helicopter bases, heli-only missions, arrive-by windows, 10 h cap as a
    constraint), one launch per algorithm; the batch's inputs (3.2 GB) are larger than L2.
    Against the oracle on one core for 256 of the instances."""
    import torch

    import oracle
    from paper_2002_11710_gb300 import api, gen

    rng = np.random.default_rng(5)
    sizes = rng.integers(12, 34, size=args.sweep_distinct)
    distinct = [gen.paper_fleet(40_000 + i, int(m)) for i, m in enumerate(sizes)]
    insts = distinct * args.sweep_copies
    B = len(insts)
    bp = api.BatchProblem(insts, dev)
    out = {"workload": (f"{B:,} paper-fleet instances ({len(distinct):,} distinct x {args.sweep_copies}), "
                        "M ~ U[12, 33], 12 vehicles (4 planes), HARD 600 min cap, arrive-by windows, "
                        "Algorithm 1 with repair, at most 100 sweeps, tenure 7"),
           "gpu_launches": 1, "timing": TIMING_BACK_TO_BACK}
    out["travel_matrix"] = run_travel_matrix(args, bp, insts, dev)
    for name, alg in (("algorithm_2", api.SWEEP_NEIGHBOURHOOD), ("algorithm_3", api.SWEEP_TABU)):
        params = api.sweep_params(100, api.HARD, 1000, 7, repair=True)
        res, _ = api.sweep_batch(bp, alg, params)
        for _ in range(max(1, args.warmup // 2)):
            api.sweep_batch(bp, alg, params, out=res)
        torch.cuda.synchronize()
        t = device_ms(lambda: api.sweep_batch(bp, alg, params, out=res))
        info = res.info.view(-1, api.INFO_LEN).cpu().numpy()
        ok = info[:, api.INFO_STATUS] == 0
        out[name] = {"ms": t, "solves_per_s": B / t * 1e3,
                     "mission_steps_per_s": float(info[ok, api.INFO_STEPS].sum()) / t * 1e3,
                     "feasible_start_frac": float(ok.mean())}
        if _env_int("RANK", 0) == 0 and args.cpu_iterations > 0:
            t0 = time.perf_counter()
            for inst in distinct[:256]:
                pb = oracle.Problem(inst, api.HARD, 1000)
                if alg == api.SWEEP_NEIGHBOURHOOD:
                    oracle.neighbourhood_search(pb, 100, repair=True)
                else:
                    oracle.tabu_sweep(pb, 7, 100, repair=True)
            dt = time.perf_counter() - t0
            out[name]["cpu_oracle"] = {"solves_per_s": 256 / dt, "cores": 1,
                                       "sample": f"first 256 distinct instances, {dt:.2f} s"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cluster", type=int, default=0, help="CTAs per cluster (0: the plan's)")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: the plan's)")
    ap.add_argument("--grid", type=int, default=0, help="clusters per instance (0: the plan's)")
    ap.add_argument("--iterations", type=int, default=0,
                    help="iterations of each single-instance search (0: the workload's; for profiling)")
    ap.add_argument("--plain-launch", action="store_true",
                    help="launch several clusters without the cooperative attribute (for ncu)")
    ap.add_argument("--cpu-iterations", type=int, default=8,
                    help="iterations of the one-core oracle sample (0 skips the CPU baselines)")
    ap.add_argument("--cpu-iterations-all", type=int, default=60,
                    help="iterations of the all-cores oracle sample")
    ap.add_argument("--ref-iterations", type=int, default=8)
    ap.add_argument("--no-paper-shaped", dest="paper_shaped", action="store_false",
                    help="skip the paper-shaped single-instance line")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 1,024-instance batched measurement")
    ap.add_argument("--no-sweeps", dest="sweeps", action="store_false",
                    help="skip the Algorithm 2 / Algorithm 3 sweep measurement")
    ap.add_argument("--sweeps-only", action="store_true",
                    help="run only the sweep measurement and print its JSON object")
    ap.add_argument("--sweep-distinct", type=int, default=16384)
    ap.add_argument("--sweep-copies", type=int, default=4)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson request stream of the serving measurement (0 skips it)")
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweeps_only:
        import torch

        torch.cuda.set_device(local_rank)
        print(json.dumps(run_sweeps(args, torch.device("cuda", local_rank))), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
