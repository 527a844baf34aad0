"""Benchmark: Tabu moves evaluated per second on the paper-shaped instance.

Workload (one "step"): one complete Tabu search of 5,000 iterations on the
paper-shaped instance (12 bases, 20 vehicles, 60 clustered facilities in a
1500 km box, 100 missions, tenure 10, duty cap 720 min as a penalty with lambda
1000), greedy start included, through asched_solve. Every iteration evaluates all
M(M+V-2) + M(M-1)/2 = 16,750 moves, so a step is 83.75 M moves.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own copy of the instance (the single-instance
search does not shard); the line reports the sum of all ranks' moves over the
slowest rank's time. `--impl reference` times the plain CPU oracle on this host's
cores instead (bounded iteration samples of the same instance).
"""
from __future__ import annotations

import argparse
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
WORKLOAD = ("paper-shaped single instance: 12 bases, 20 vehicles, 60 facilities in 4 Gaussian "
            "clusters (sigma 80 km) + 20% uniform outliers in a 1500 km box, 100 uniform missions, "
            "int32 minutes at 250 km/h, duty cap 720 min (penalty, lambda 1000), tenure 10, "
            "5,000 iterations, greedy start")
# Algorithmic int32 operations per evaluated move (see the roofline section of the
# design notes): a relocation is 23 ops, a swap 34, mixed in proportion.
OPS_RELOCATE = 23
OPS_SWAP = 34
# DRAM bytes (read + write) of one solve launch, from the ncu capture summarised in
# profiles/tabu_kernel_paper_shaped.md. Valid only for the kernel source it was taken
# on; any other source reports traffic as null.
TRAFFIC_BYTES = 126976
TRAFFIC_SOURCE_SHA = "0271976a8fe2d5c8"


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


def traffic_bytes():
    src = os.path.join(ROOT, "paper_2002_11710_gb300", "csrc", "asched.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    return TRAFFIC_BYTES if sha == TRAFFIC_SOURCE_SHA else None


def moves_split(M, V):
    return M * (M + V - 2), M * (M - 1) // 2


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


def cpu_oracle_sample(inst, p, iterations):
    """The oracle as it stands, one core, on the first `iterations` iterations."""
    import oracle

    pb = oracle.Problem(inst, p.cap_mode, p.lam)
    t0 = time.perf_counter()
    r = oracle.tabu_search(pb, p.tenure, iterations)
    dt = time.perf_counter() - t0
    assert r["status"] == 0
    M, V = inst.n_missions, inst.n_vehicles
    n = (M * (M + V - 2) + M * (M - 1) // 2) * iterations
    return n / dt, dt


def max_over_ranks(seconds, world, device):
    """The slowest rank's time (all ranks call this; world 1 returns the input)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args, rank, world):
    from paper_2002_11710_gb300 import gen

    if rank != 0:
        return
    inst, p = gen.paper_shaped(0), gen.PAPER_SHAPED_PARAMS
    it_sample = args.ref_iterations
    for _ in range(args.warmup):
        cpu_oracle_sample(inst, p, it_sample)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = cpu_oracle_sample(inst, p, it_sample)
        rates.append(r)
        times.append(dt)
    M, V = inst.n_missions, inst.n_vehicles
    n = (M * (M + V - 2) + M * (M - 1) // 2) * it_sample
    value = n * len(times) / sum(times)
    sample = f"first {it_sample} of 5,000 iterations of the paper-shaped instance per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample, "n_missions": M, "n_vehicles": V},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2002_11710_gb300 import api, gen

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    inst, p = gen.paper_shaped(0), gen.PAPER_SHAPED_PARAMS
    M, V = inst.n_missions, inst.n_vehicles
    R, S = moves_split(M, V)
    moves_step = (R + S) * p.iterations
    params = api.params_from(p, cluster_size=args.cluster, block_threads=args.threads)
    dp = api.DeviceProblem(inst, dev)
    plan = api.plan(dp, params)
    out = api.alloc_output(dp, p.iterations)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up (also checks the device status)
    for _ in range(args.warmup):
        api.solve(dp, params, out=out)
    torch.cuda.synchronize()
    info = out.info.cpu().numpy()
    if info[api.INFO_STATUS] != 0:
        raise RuntimeError(f"device status {info[api.INFO_STATUS]}")
    z_best = int(info[api.INFO_Z_BEST])

    clocks = Clocks(local_rank) if rank == 0 else None
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
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(step_ms) / 1000.0
    clk = clocks.stop() if clocks else None
    dev_s = max_over_ranks(dev_s, world, dev)
    # end to end through the public API from host data
    pinned = api.pin_instance(inst)
    e2e_times = []
    h2d = pinned.nbytes()
    d2h = 0
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
    e2e_s = sum(e2e_times)
    e2e_s = max_over_ranks(e2e_s, world, dev)
    batched = run_batched(args, dev) if args.batched else None
    serving = run_serving(args, dev) if args.serve_seconds > 0 else None
    sweeps = run_sweeps(args, dev) if args.sweeps else None
    if rank != 0:
        return
    value = whole_job_rate(moves_step * args.steps, world, dev_s)
    e2e_value = whole_job_rate(moves_step * args.steps, world, e2e_s)
    launch_s = statistics.mean(step_ms) / 1000.0
    ops = (R * OPS_RELOCATE + S * OPS_SWAP) * p.iterations
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    int_lanes = args.int32_lanes_per_sm
    peak_tops = sm_count * int_lanes * sm_max_mhz * 1e6 / 1e12
    achieved = ops / launch_s / 1e12
    cpu_rate, cpu_dt = cpu_oracle_sample(inst, p, args.cpu_iterations) if args.cpu_iterations > 0 else (None, 0)
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_missions": M, "n_vehicles": V,
                   "iterations": p.iterations, "moves_per_iteration": R + S,
                   "moves_per_step": moves_step, "cluster_size": plan.cluster_size,
                   "block_threads": plan.block_threads, "smem_bytes": plan.smem_bytes,
                   "l2": "flushed between steps (256 MB write, untimed)",
                   "parallelism": "one instance per GPU (replicas)"},
        "solves_per_s": world * args.steps / dev_s,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "wall_s": wall,
        "z_best": z_best,
        "gpu_launches": args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved / peak_tops, "traffic": traffic_bytes(),
                     "peak_basis": f"{sm_count} SMs x {int_lanes} int32 lanes/clk x {sm_max_mhz:.0f} MHz",
                     "frac_of_sms_used": achieved / (peak_tops * plan.cluster_size / sm_count)},
        "batched": batched,
        "serving": serving,
        "sweeps": sweeps,
        "cpu_baseline": None if cpu_rate is None else {
            "value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {args.cpu_iterations} of 5,000 iterations, same instance, {cpu_dt:.1f} s"},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_batched(args, dev):
    """The batched workload: 1,024 instances (V ~ U[3, 30], M ~ U[10, 200], paper-shaped
    geography, 2,000 iterations each) in one persistent launch, block size picked by the
    autotuner, against the same instances as 1,024 single-instance launches."""
    import torch

    from paper_2002_11710_gb300 import api, gen

    insts = [gen.batched_member(i) for i in range(1024)]
    p = gen.BATCHED_PARAMS
    moves = sum(api.num_moves(i.n_missions, i.n_vehicles) for i in insts) * p.iterations
    bp = api.BatchProblem(insts, dev)
    choice, tune = api.autotune_batch(bp, api.params_from(p))
    params = api.tuned_params(api.params_from(p), choice)
    thr = {"block_threads": choice[0], "layout": "int16 matrix" if choice[1] else "gather tables"}
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
    seq_ms = a.elapsed_time(b)
    t = statistics.median(ms)
    return {"workload": "1,024 instances, V ~ U[3,30], M ~ U[10,200], 2,000 iterations each, "
                        "replayed from a captured CUDA graph",
            "ms": t, "solves_per_s": 1024 / t * 1e3, "moves_per_s": moves / t * 1e3,
            "launch_shape": thr, "autotune_ms": {f"{t}{'/int16' if c else ''}": v for (t, c), v in tune.items()},
            "instances_ok": ok,
            "sequential_ms": seq_ms, "sequential_solves_per_s": 1024 / seq_ms * 1e3,
            "speedup_vs_sequential": seq_ms / t, "gpu_launches": 2}


# Requests of at least BIG_MISSIONS missions go to a launch of BIG_CLUSTERS clusters of
# BIG_CLUSTER CTAs (chosen by a sweep on this stream: p99 27.1 ms with one-CTA workers
# only, 5.0 ms with this lane).
BIG_MISSIONS, BIG_CLUSTER, BIG_CLUSTERS = 60, 8, 8


def run_serving(args, dev):
    """The serving workload: Poisson re-planning requests at 2,000 req/s (sizes
    lognormal around 60 missions, clipped to [10, 400], V = ceil(M/5), 1,000 iterations
    each) through the continuous-batching server, with slots admitted under a 40 GB
    device-memory budget; against the plain path (one asched_solve launch per request,
    in arrival order on one stream) for the first second of the same stream."""
    import torch

    from paper_2002_11710_gb300 import api, gen, serve

    params = api.params_from(gen.SERVING_PARAMS)
    pool = [gen.serving_request(20_000 + k) for k in range(2048)]
    arrivals = gen.poisson_arrivals(7, 2000.0, args.serve_seconds)
    reqs = [pool[k % len(pool)] for k in range(len(arrivals))]
    srv = serve.Server(max_loc=72, max_vehicles=80, max_missions=400, n_slots=4096,
                       budget_bytes=40 << 30, device=dev, big_missions=BIG_MISSIONS,
                       big_cluster=BIG_CLUSTER, big_clusters=BIG_CLUSTERS)
    srv.start(params, idle_timeout_s=60.0)
    try:
        lat, wall = serve.run_stream(srv, reqs, arrivals)
    finally:
        srv.stop()
    served = srv.served()
    # plain per-request path on the first second of arrivals
    n_plain = int((arrivals < 1.0).sum())
    dps = [api.DeviceProblem(r, dev) for r in reqs[:n_plain]]
    outs = [api.alloc_output(d, params.iterations) for d in dps]
    torch.cuda.synchronize()
    st = torch.cuda.Stream(device=dev)
    evs = [torch.cuda.Event() for _ in range(n_plain)]
    lat2 = np.zeros(n_plain)
    t0 = time.perf_counter()
    i = k = 0
    while k < n_plain:
        now = time.perf_counter() - t0
        while i < n_plain and arrivals[i] <= now:
            api.solve(dps[i], params, out=outs[i], stream=st)
            evs[i].record(st)
            i += 1
        while k < i and evs[k].query():
            lat2[k] = time.perf_counter() - t0 - arrivals[k]
            k += 1
    wall2 = time.perf_counter() - t0
    return {"workload": (f"Poisson 2,000 req/s for {args.serve_seconds:g} s, M ~ lognormal(median 60) "
                         "in [10, 400], V = ceil(M/5), 1,000 iterations, 40 GB slot budget"),
            "lanes": {"one_cta": f"requests of fewer than {BIG_MISSIONS} missions, one CTA each",
                      "clusters": f"requests of {BIG_MISSIONS} missions or more, {BIG_CLUSTERS} clusters "
                                  f"of {BIG_CLUSTER} CTAs, one cluster per request"},
            "requests": len(reqs), "served": served, "wall_s": wall,
            "solves_per_s": len(reqs) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                           "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(lat.max() * 1e3)},
            "slots": srv.n_slots, "slot_bytes": srv.slot_bytes,
            "plain_per_request": {"requests": n_plain, "solves_per_s": n_plain / wall2,
                                  "latency_ms": {"p50": float(np.percentile(lat2, 50) * 1e3),
                                                 "p99": float(np.percentile(lat2, 99) * 1e3)}}}


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
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f).get("hbm_gbs"))
    except (OSError, TypeError, ValueError):
        pass
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
            res[name]["frac_of_measured_hbm"] = nbytes / t / 1e6 / hbm
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
                     "feasible_start_frac": float(ok.mean()),
                     "mean_sweeps": float(info[ok, api.INFO_ITERS].mean()),
                     "mean_improvement_pct": float(100.0 * (1.0 - info[ok, api.INFO_Z_BEST].sum() /
                                                              info[ok, api.INFO_Z_INIT].sum()))}
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
    out["multi_start"] = run_multi_start(args, distinct, res, dev)
    out["single_instance"] = run_sweep_latency(dev)
    return out


# The paper's per-instance runtimes (seconds; Python + Numba on an i9-7920X, its CUDA
# variants on a GTX 1080 Ti), its Table 1, by number of missions: context, not a target.
PAPER_RUNTIME_S = {
    12: {"ns": 0.0153, "ns_cuda": 0.548, "tabu": 0.0245, "tabu_cuda": 0.578},
    15: {"ns": 0.0244, "ns_cuda": 0.532, "tabu": 0.0349, "tabu_cuda": 0.615},
    18: {"ns": 0.0322, "ns_cuda": 0.544, "tabu": 0.0424, "tabu_cuda": 0.575},
    21: {"ns": 0.0446, "ns_cuda": 0.519, "tabu": 0.0553, "tabu_cuda": 0.507},
    24: {"ns": 0.0499, "ns_cuda": 0.611, "tabu": 0.0618, "tabu_cuda": 0.642},
    27: {"ns": 0.0565, "ns_cuda": 0.618, "tabu": 0.0675, "tabu_cuda": 0.561},
    30: {"ns": 0.0581, "ns_cuda": 0.599, "tabu": 0.0682, "tabu_cuda": 0.645},
    33: {"ns": 0.0631, "ns_cuda": 0.686, "tabu": 0.0689, "tabu_cuda": 0.611},
}


def run_sweep_latency(dev):
    """One paper-fleet instance per launch at the paper's sizes (12-33 missions, its fleet),
    Algorithm 2 and Algorithm 3 (tenure 7), repair on, HARD cap: device time per solve
    (CUDA events around the launch, median of 20), beside the paper's own runtimes."""
    import torch

    from paper_2002_11710_gb300 import api, gen

    res = {}
    for m in sorted(PAPER_RUNTIME_S):
        inst = gen.paper_fleet(90_000 + m, m)
        bp = api.BatchProblem([inst], dev)
        row = {"paper_s": PAPER_RUNTIME_S[m]}
        for name, alg in (("algorithm_2_ms", api.SWEEP_NEIGHBOURHOOD), ("algorithm_3_ms", api.SWEEP_TABU)):
            params = api.sweep_params(100, api.HARD, 1000, 7, repair=True)
            out, _ = api.sweep_batch(bp, alg, params)
            torch.cuda.synchronize()
            ts = []
            for _ in range(20):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                api.sweep_batch(bp, alg, params, out=out)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            row[name] = statistics.median(ts)
            row["status"] = int(out.info[api.INFO_STATUS].item())
        res[str(m)] = row
    return res


def run_multi_start(args, distinct, default_res, dev):
    """The paper's repeated runs (it reports best, worst and mean of 10 runs whose loop
    orders are random permutations): 16 runs of Algorithm 3 (tenure 7, repair) for each
    of the first 4,096 paper-fleet instances, each run with its own seeded vehicle order
    and mission ranks, all 65,536 runs in one launch. Quality: best of 16 against the
    run in index order (from the batch above, same instances and parameters)."""
    import torch

    from paper_2002_11710_gb300 import api, gen

    R = 16
    base = distinct[:4096]
    insts = [inst for inst in base for _ in range(R)]
    orders = [gen.sweep_orders(70_000 + k, inst.n_vehicles, inst.n_missions) for k, inst in enumerate(insts)]
    bp = api.BatchProblem(insts, dev)
    ords = api.sweep_orders_tensors(bp, orders)
    params = api.sweep_params(100, api.HARD, 1000, 7, repair=True)
    res, _ = api.sweep_batch(bp, api.SWEEP_TABU, params, orders=ords)
    torch.cuda.synchronize()
    t_ms = device_ms(lambda: api.sweep_batch(bp, api.SWEEP_TABU, params, out=res, orders=ords))
    info = res.info.view(len(base), R, api.INFO_LEN).cpu().numpy()
    ok = info[:, :, api.INFO_STATUS] == 0
    z = np.where(ok, info[:, :, api.INFO_Z_BEST], np.iinfo(np.int32).max).astype(np.int64)
    d0 = default_res.info.view(-1, api.INFO_LEN)[:len(base)].cpu().numpy()
    both = ok.any(axis=1) & (d0[:, api.INFO_STATUS] == 0)
    best = z.min(axis=1)
    zz = np.where(ok, z, 0)
    n_ok = np.maximum(ok.sum(axis=1), 1)
    mean = zz.sum(axis=1) / n_ok
    worst = np.where(ok, z, 0).max(axis=1)
    t = t_ms
    return {"workload": "4,096 paper-fleet instances x 16 runs with seeded random loop orders, "
                        "Algorithm 3 (tenure 7, repair), one launch",
            "ms": t, "runs_per_s": len(insts) / t * 1e3, "instances_per_s": len(base) / t * 1e3,
            "runs_feasible_frac": float(ok.mean()),
            "instances_feasible_any_run": float(ok.any(axis=1).mean()),
            "instances_feasible_index_order": float((d0[:, api.INFO_STATUS] == 0).mean()),
            "best_of_16_vs_index_order_pct": float(100.0 * (1.0 - best[both].sum() / d0[both, api.INFO_Z_BEST].sum())),
            "mean_worst_minus_best_pct": float(100.0 * np.mean((worst[both] - best[both]) / best[both])),
            "mean_mean_minus_best_pct": float(100.0 * np.mean((mean[both] - best[both]) / best[both])),
            "gpu_launches": 1, "timing": TIMING_BACK_TO_BACK}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--cpu-iterations", type=int, default=600)
    ap.add_argument("--ref-iterations", type=int, default=100)
    ap.add_argument("--int32-lanes-per-sm", type=int, default=128)
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 1,024-instance batched measurement")
    ap.add_argument("--no-sweeps", dest="sweeps", action="store_false",
                    help="skip the Algorithm 2 / Algorithm 3 sweep measurement")
    ap.add_argument("--sweeps-only", action="store_true",
                    help="run only the sweep measurement and print its JSON object")
    ap.add_argument("--sweep-distinct", type=int, default=16384)
    ap.add_argument("--sweep-copies", type=int, default=4)
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="length of the Poisson request stream for the serving measurement "
                         "(the serving workload is 60 s; 0 skips it)")
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
