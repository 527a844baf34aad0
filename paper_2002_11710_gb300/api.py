"""Python binding of the C ABI (include/asched.h), with PyTorch owning device memory.

Every function marshals arguments and calls the library; all computation of the
search runs in the library's CUDA kernels. PyTorch provides device memory and the
current stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (COMPACT_LAYOUT, E_CUDA, E_INFEASIBLE_INIT, E_INVALID, E_OVERFLOW_GUARD, E_TIMEOUT,  # noqa: F401
                   E_TOO_LARGE, FLAG_ADMISSIBLE, FLAG_ASPIRATION, FLAG_FEASIBLE, FLAG_TABU, HARD,
                   INFO_BEST_IT, INFO_ITERS, INFO_LEN, INFO_STATUS, INFO_Z_BEST, INFO_Z_FINAL,
                   INFO_Z_INIT, NULL_MOVE, OK, PENALTY, SWAP_BIT, AschedError)
from ._lib import INFO_MOVES, INFO_STEPS, SWEEP_ACCEPT_WORSE, SWEEP_NEIGHBOURHOOD, SWEEP_REPAIR, SWEEP_TABU  # noqa: F401


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def num_moves(n_missions: int, n_vehicles: int) -> int:
    out = ctypes.c_int64(0)
    _lib.check(_lib.load().asched_num_moves(int(n_missions), int(n_vehicles), ctypes.byref(out)),
               "asched_num_moves")
    return int(out.value)


def make_params(tenure: int, iterations: int, cap_mode: int = HARD, lam: int = 1000,
                cluster_size: int = 0, block_threads: int = 0, timeout_ns: int = 0,
                compact: bool = False, grid_clusters: int = 0, plain_launch: bool = False) -> _lib.Params:
    """compact: keep the travel matrix as int16 in shared memory instead of the gather
    tables (used automatically when the tables do not fit). grid_clusters: clusters
    cooperating on one instance (0 = automatic). plain_launch: launch several clusters
    without the cooperative attribute (for profilers)."""
    flags = (_lib.COMPACT_LAYOUT if compact else 0) | (_lib.PLAIN_LAUNCH if plain_launch else 0)
    return _lib.Params(int(tenure), int(iterations), int(cap_mode), int(lam), int(cluster_size),
                       int(block_threads), int(timeout_ns), flags, int(grid_clusters))


def params_from(p, **overrides) -> _lib.Params:
    """ctypes parameters from a gen.Params-like object (tenure, iterations, cap_mode, lam)."""
    kw = dict(tenure=p.tenure, iterations=p.iterations, cap_mode=p.cap_mode, lam=p.lam)
    kw.update(overrides)
    return make_params(**kw)


def _i32(a, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=torch.int32, non_blocking=True)
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32))
    return t.to(device, non_blocking=True)


@dataclasses.dataclass
class PinnedInstance:
    """An instance's arrays in pinned host memory, ready for asynchronous upload."""
    travel: torch.Tensor
    veh_base: torch.Tensor
    veh_type: torch.Tensor
    pickup: torch.Tensor
    delivery: torch.Tensor
    heli_only: Optional[torch.Tensor]
    deadline: Optional[torch.Tensor]
    duty_cap: int
    horizon: int

    def nbytes(self) -> int:
        return sum(int(t.numel()) * 4 for t in (self.travel, self.veh_base, self.veh_type,
                                                 self.pickup, self.delivery, self.heli_only,
                                                 self.deadline) if t is not None)


def pin_instance(inst) -> PinnedInstance:
    def pin(a):
        if a is None:
            return None
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).pin_memory()

    return PinnedInstance(pin(inst.travel), pin(inst.veh_base), pin(inst.veh_type),
                          pin(inst.pickup), pin(inst.delivery), pin(inst.heli_only),
                          pin(inst.deadline), int(inst.duty_cap), int(inst.horizon))


class DeviceProblem:
    """An instance resident in device memory (int32 torch tensors) and its C struct.

    `inst` is any object with the fields of gen.Instance (travel, veh_base, veh_type,
    pickup, delivery, heli_only, deadline, duty_cap, horizon).
    """

    def __init__(self, inst, device="cuda"):
        self.device = torch.device(device)
        self.n_loc = int(inst.travel.shape[1])
        self.n_types = int(inst.travel.shape[0])
        self.V = int(len(inst.veh_base))
        self.M = int(len(inst.pickup))
        self.duty_cap = int(inst.duty_cap)
        self.horizon = int(inst.horizon)
        dev = self.device
        self.travel = _i32(inst.travel, dev)
        self.veh_base = _i32(inst.veh_base, dev)
        self.veh_type = _i32(inst.veh_type, dev)
        self.pickup = _i32(inst.pickup if self.M else np.zeros(1, np.int32), dev)
        self.delivery = _i32(inst.delivery if self.M else np.zeros(1, np.int32), dev)
        self.heli_only = None if inst.heli_only is None else _i32(inst.heli_only, dev)
        self.deadline = None if inst.deadline is None else _i32(inst.deadline, dev)
        self.struct = self._struct()
        self._ws = None
        self._ws_bytes = {}  # asched_workspace_bytes by params

    def workspace(self, nbytes: int) -> Optional[torch.Tensor]:
        """Device workspace of at least nbytes for asched_tabu_solve (kept and reused;
        None when nbytes is 0). Two searches of this problem in flight at once on
        different streams need their own workspaces."""
        if nbytes <= 0:
            return None
        if self._ws is None or self._ws.numel() * 8 < nbytes:
            self._ws = torch.zeros((nbytes + 7) // 8, dtype=torch.int64, device=self.device)
        return self._ws

    def _struct(self):
        return _lib.Instance(self.n_loc, self.n_types, self.V, self.M, _ptr(self.travel),
                             _ptr(self.veh_base), _ptr(self.veh_type), _ptr(self.pickup),
                             _ptr(self.delivery), _ptr(self.heli_only), _ptr(self.deadline),
                             self.duty_cap, self.horizon)


def host_struct(inst):
    """C struct over HOST numpy arrays (for asched_check_instance_host); keep the
    returned arrays alive while the struct is used."""
    keep = [np.ascontiguousarray(inst.travel, dtype=np.int32),
            np.ascontiguousarray(inst.veh_base, dtype=np.int32),
            np.ascontiguousarray(inst.veh_type, dtype=np.int32),
            np.ascontiguousarray(inst.pickup, dtype=np.int32),
            np.ascontiguousarray(inst.delivery, dtype=np.int32),
            None if inst.heli_only is None else np.ascontiguousarray(inst.heli_only, dtype=np.int32),
            None if inst.deadline is None else np.ascontiguousarray(inst.deadline, dtype=np.int32)]

    def hp(a):
        return None if a is None else ctypes.c_void_p(a.ctypes.data)

    s = _lib.Instance(int(keep[0].shape[1]), int(keep[0].shape[0]), int(keep[1].shape[0]),
                      int(keep[3].shape[0]), *[hp(a) for a in keep], int(inst.duty_cap),
                      int(inst.horizon))
    return s, keep


def check_instance_host(inst, params: _lib.Params) -> int:
    s, keep = host_struct(inst)
    return int(_lib.load().asched_check_instance_host(ctypes.byref(s), ctypes.byref(params)))


def workspace_bytes(dp: DeviceProblem, params: _lib.Params) -> int:
    n = ctypes.c_size_t(0)
    _lib.check(_lib.load().asched_workspace_bytes(ctypes.byref(dp.struct), ctypes.byref(params), ctypes.byref(n)),
               "asched_workspace_bytes")
    return int(n.value)


def plan(dp: DeviceProblem, params: _lib.Params) -> _lib.Plan:
    out = _lib.Plan()
    _lib.check(_lib.load().asched_plan(ctypes.byref(dp.struct), ctypes.byref(params),
                                       ctypes.byref(out)), "asched_plan")
    return out


@dataclasses.dataclass
class SolveOutput:
    """Device tensors written by asched_solve (valid after the stream is synchronised)."""
    route_off: torch.Tensor
    route: torch.Tensor
    flight: torch.Tensor
    overflow: torch.Tensor
    info: torch.Tensor
    traj_move: Optional[torch.Tensor]
    traj_z: Optional[torch.Tensor]

    def struct(self):
        return _lib.Result(_ptr(self.route_off), _ptr(self.route), _ptr(self.flight),
                           _ptr(self.overflow), _ptr(self.info), _ptr(self.traj_move),
                           _ptr(self.traj_z))


def alloc_output(dp: DeviceProblem, iterations: int, trajectory: bool = False) -> SolveOutput:
    dev = dp.device

    def z(n):
        return torch.zeros(max(n, 1), dtype=torch.int32, device=dev)

    return SolveOutput(route_off=z(dp.V + 1), route=z(dp.M), flight=z(dp.V), overflow=z(dp.V),
                       info=z(INFO_LEN), traj_move=z(iterations) if trajectory else None,
                       traj_z=z(iterations) if trajectory else None)


def solve(dp: DeviceProblem, params: _lib.Params, init=None, out: Optional[SolveOutput] = None,
          trajectory: bool = False, stream: Optional[torch.cuda.Stream] = None,
          workspace: Optional[torch.Tensor] = None) -> SolveOutput:
    """Queue one Tabu search (asched_tabu_solve, on the launch shape of asched_plan) on
    `stream` (default: torch's current stream).

    init: None (greedy start, Algorithm 1) or (route_off, route) device int32 tensors.
    workspace: device tensor for the keys between clusters (default: the problem's own,
    sized by asched_workspace_bytes). Returns the output tensors; read them after
    synchronising the stream.
    """
    if out is None:
        out = alloc_output(dp, params.iterations, trajectory)
    s = stream if stream is not None else torch.cuda.current_stream(dp.device)
    res = out.struct()
    ioff, iroute = (None, None) if init is None else (_ptr(init[0]), _ptr(init[1]))
    if workspace is None:
        key = bytes(params)
        nb = dp._ws_bytes.get(key)
        if nb is None:
            nb = dp._ws_bytes[key] = workspace_bytes(dp, params)
        workspace = dp.workspace(nb)
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = _lib.load().asched_tabu_solve(ctypes.byref(dp.struct), ctypes.byref(params), ioff, iroute,
                                       ctypes.byref(res), _ptr(workspace), ctypes.c_size_t(nbytes),
                                       ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_tabu_solve")
    return out


def solve_one_cluster(dp: DeviceProblem, params: _lib.Params, init=None, out: Optional[SolveOutput] = None,
                      trajectory: bool = False, stream: Optional[torch.cuda.Stream] = None) -> SolveOutput:
    """Queue asched_solve: the same search on one cluster, with no workspace."""
    if out is None:
        out = alloc_output(dp, params.iterations, trajectory)
    s = stream if stream is not None else torch.cuda.current_stream(dp.device)
    res = out.struct()
    ioff, iroute = (None, None) if init is None else (_ptr(init[0]), _ptr(init[1]))
    rc = _lib.load().asched_solve(ctypes.byref(dp.struct), ctypes.byref(params), ioff, iroute,
                                  ctypes.byref(res), ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_solve")
    return out


def greedy_init(dp: DeviceProblem, params: _lib.Params, stream: Optional[torch.cuda.Stream] = None):
    """Algorithm 1 alone on the device (asched_greedy_init): (route_off, route, info)
    device tensors; read them after synchronising the stream."""
    z = lambda n: torch.zeros(max(n, 1), dtype=torch.int32, device=dp.device)  # noqa: E731
    off, route, info = z(dp.V + 1), z(dp.M), z(INFO_LEN)
    s = stream if stream is not None else torch.cuda.current_stream(dp.device)
    rc = _lib.load().asched_greedy_init(ctypes.byref(dp.struct), ctypes.byref(params), _ptr(off), _ptr(route),
                                        _ptr(info), ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_greedy_init")
    return off, route, info


def eval_neighbourhood(dp: DeviceProblem, params: _lib.Params, route_off: torch.Tensor,
                       route: torch.Tensor, tabu_until: Optional[torch.Tensor], it: int,
                       z_best: int, with_ids: bool = True,
                       stream: Optional[torch.cuda.Stream] = None):
    """Queue asched_eval_neighbourhood; returns (delta, flags, ids or None, best_key, info)."""
    n = num_moves(dp.M, dp.V)
    dev = dp.device
    delta = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    flags = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
    ids = torch.zeros(max(n, 1), dtype=torch.int32, device=dev) if with_ids else None
    key = torch.zeros(1, dtype=torch.int64, device=dev)
    info = torch.zeros(INFO_LEN, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = _lib.load().asched_eval_neighbourhood(
        ctypes.byref(dp.struct), ctypes.byref(params), _ptr(route_off), _ptr(route),
        _ptr(tabu_until), int(it), int(z_best), _ptr(delta), _ptr(flags), _ptr(ids), _ptr(key),
        _ptr(info), ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_eval_neighbourhood")
    return delta[:n], flags[:n], (ids[:n] if ids is not None else None), key, info


def solve_host(inst, params: _lib.Params, trajectory: bool = False, device="cuda",
               stream: Optional[torch.cuda.Stream] = None):
    """End-to-end call for host data: host -> device copies of the instance (pass a
    PinnedInstance for asynchronous copies from pinned memory), one asched_solve,
    device -> host copies of the result, then a synchronise.
    Returns numpy arrays and the info words."""
    dev = torch.device(device)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(s):
        dp = DeviceProblem(inst, dev)
        out = solve(dp, params, trajectory=trajectory, stream=s)
        host = {k: getattr(out, k).to("cpu", non_blocking=True)
                for k in ("route_off", "route", "flight", "overflow", "info")}
        if trajectory:
            host["traj_move"] = out.traj_move.to("cpu", non_blocking=True)
            host["traj_z"] = out.traj_z.to("cpu", non_blocking=True)
    s.synchronize()
    res = {k: v.numpy() for k, v in host.items()}
    res["route"] = res["route"][: dp.M]
    if trajectory:
        res["traj_move"] = res["traj_move"][: params.iterations].view(np.uint32)
        res["traj_z"] = res["traj_z"][: params.iterations]
    return res


# ------------------------------------------------------------------------- batches --

class BatchProblem:
    """Many instances packed into concatenated device arrays (the asched_batch layout).

    All instances must have the same number of travel layers, and either all or none
    have deadlines (heli-only flags may be missing on some: they count as 0)."""

    def __init__(self, instances, device="cuda"):
        self.device = torch.device(device)
        insts = list(instances)
        self.B = len(insts)
        nt = {int(i.travel.shape[0]) for i in insts}
        if len(nt) > 1:
            raise ValueError("every instance needs the same number of travel layers")
        self.n_types = nt.pop() if insts else 1
        dl = {i.deadline is not None for i in insts}
        if len(dl) > 1:
            raise ValueError("either every instance has deadlines or none has")
        self.has_deadlines = bool(dl and dl.pop())
        L = np.array([i.travel.shape[1] for i in insts], np.int64)
        V = np.array([len(i.veh_base) for i in insts], np.int64)
        M = np.array([len(i.pickup) for i in insts], np.int64)
        self.h_loc_off = np.concatenate([[0], np.cumsum(L)]).astype(np.int32)
        self.h_veh_off = np.concatenate([[0], np.cumsum(V)]).astype(np.int32)
        self.h_mis_off = np.concatenate([[0], np.cumsum(M)]).astype(np.int32)
        tsz = self.n_types * L * L
        self.h_travel_off = np.concatenate([[0], np.cumsum(tsz)])[:-1].astype(np.int64)

        def cat(arrs, dtype=np.int32):
            arrs = [np.ascontiguousarray(a, dtype=dtype).reshape(-1) for a in arrs]
            out = np.concatenate(arrs) if arrs else np.zeros(0, dtype)
            return out if out.size else np.zeros(1, dtype)

        dev = self.device
        t = lambda a, dt=torch.int32: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)  # noqa: E731
        self.loc_off = t(self.h_loc_off)
        self.veh_off = t(self.h_veh_off)
        self.mis_off = t(self.h_mis_off)
        self.travel_off = t(self.h_travel_off if self.B else np.zeros(1, np.int64), torch.int64)
        self.travel = t(cat([i.travel for i in insts]))
        self.veh_base = t(cat([i.veh_base for i in insts]))
        self.veh_type = t(cat([i.veh_type for i in insts]))
        self.pickup = t(cat([i.pickup for i in insts]))
        self.delivery = t(cat([i.delivery for i in insts]))
        any_heli = any(i.heli_only is not None for i in insts)
        self.heli_only = t(cat([i.heli_only if i.heli_only is not None else np.zeros(len(i.pickup))
                                for i in insts])) if any_heli else None
        self.deadline = t(cat([i.deadline for i in insts])) if self.has_deadlines else None
        self.duty_cap = t(np.array([i.duty_cap for i in insts] or [0], np.int32))
        self.horizon = t(np.array([i.horizon for i in insts] or [0], np.int32))
        ws = ctypes.c_size_t(0)
        _lib.check(_lib.load().asched_batch_workspace_bytes(self.B, ctypes.byref(ws)),
                   "asched_batch_workspace_bytes")
        self.workspace = torch.zeros((ws.value + 3) // 4, dtype=torch.int32, device=dev)
        hp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        self.struct = _lib.Batch(self.B, self.n_types, hp(self.h_loc_off), hp(self.h_veh_off),
                                 hp(self.h_mis_off), _ptr(self.loc_off), _ptr(self.veh_off),
                                 _ptr(self.mis_off), _ptr(self.travel_off), _ptr(self.travel),
                                 _ptr(self.veh_base), _ptr(self.veh_type), _ptr(self.pickup),
                                 _ptr(self.delivery), _ptr(self.heli_only), _ptr(self.deadline),
                                 _ptr(self.duty_cap), _ptr(self.horizon))

    def alloc_output(self):
        dev = self.device
        nv = int(self.h_veh_off[-1])
        nm = int(self.h_mis_off[-1])
        z = lambda n: torch.zeros(max(n, 1), dtype=torch.int32, device=dev)  # noqa: E731
        return BatchOutput(route_off=z(nv + self.B), route=z(nm), flight=z(nv), overflow=z(nv),
                           info=z(self.B * INFO_LEN))

    def unpack(self, out: "BatchOutput", b: int):
        """Instance b's results as numpy arrays (call after synchronising)."""
        vo, v1 = int(self.h_veh_off[b]), int(self.h_veh_off[b + 1])
        mo, m1 = int(self.h_mis_off[b]), int(self.h_mis_off[b + 1])
        return {"route_off": out.route_off[vo + b: v1 + b + 1].cpu().numpy(),
                "route": out.route[mo:m1].cpu().numpy(),
                "flight": out.flight[vo:v1].cpu().numpy(),
                "overflow": out.overflow[vo:v1].cpu().numpy(),
                "info": out.info[b * INFO_LEN:(b + 1) * INFO_LEN].cpu().numpy()}


@dataclasses.dataclass
class BatchOutput:
    route_off: torch.Tensor
    route: torch.Tensor
    flight: torch.Tensor
    overflow: torch.Tensor
    info: torch.Tensor

    def struct(self):
        return _lib.BatchResult(_ptr(self.route_off), _ptr(self.route), _ptr(self.flight),
                                _ptr(self.overflow), _ptr(self.info))


def solve_batch(bp: BatchProblem, params: _lib.Params, out: Optional[BatchOutput] = None,
                stream: Optional[torch.cuda.Stream] = None) -> BatchOutput:
    """Queue asched_solve_batch on `stream` (default: torch's current stream)."""
    if out is None:
        out = bp.alloc_output()
    s = stream if stream is not None else torch.cuda.current_stream(bp.device)
    res = out.struct()
    rc = _lib.load().asched_solve_batch(ctypes.byref(bp.struct), ctypes.byref(params),
                                        ctypes.byref(res), _ptr(bp.workspace),
                                        ctypes.c_size_t(bp.workspace.numel() * 4),
                                        ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_solve_batch")
    return out


BATCH_CANDIDATES = ((512, False, 1), (384, False, 1), (256, False, 1), (256, True, 1), (128, True, 1),
                    (512, False, 2), (256, False, 2), (512, False, 4))


def _shape(cand):
    """(block threads, compact, CTAs per instance) of an autotune candidate given as a
    block size, a (threads, compact) pair or a full triple."""
    if isinstance(cand, int):
        return int(cand), False, 1
    if len(cand) == 2:
        return int(cand[0]), bool(cand[1]), 1
    return int(cand[0]), bool(cand[1]), int(cand[2])


def batch_moves_per_warp(bp: "BatchProblem", cand) -> float:
    """Moves each warp evaluates per iteration, averaged over the batch's instances, for
    an autotune candidate: the neighbourhood over the warps of the CTAs that solve one
    instance (the moves-per-warp axis the block size and CTAs per instance set)."""
    thr, _, cl = _shape(cand)
    moves = [num_moves(int(m), int(v)) for m, v in zip(np.diff(bp.h_mis_off), np.diff(bp.h_veh_off))]
    return float(np.mean(moves)) / (thr // 32 * cl) if moves else 0.0


def autotune_batch(bp: BatchProblem, params: _lib.Params, candidates=BATCH_CANDIDATES,
                   probe_iterations: int = 200, repeats: int = 2):
    """Pick the launch shape of a batch by timing short probe runs of each candidate
    (CUDA events on the current stream). A candidate is (block threads, compact, CTAs per
    instance): compact means the int16 matrix layout for every instance (smaller state,
    more resident CTAs) instead of the gather tables where they fit; CTAs per instance > 1
    solves each instance by a thread-block cluster of that many CTAs. Block size and CTAs
    per instance together set the moves each warp evaluates (batch_moves_per_warp). A
    plain int is a block size, a pair (threads, compact) has one CTA per instance.
    Results never depend on the choice; only the time does. Returns (best candidate,
    {candidate: ms}) with candidates as triples; shapes the device cannot launch (a
    cluster that does not fit) are left out."""
    out = bp.alloc_output()
    times = {}
    for cand in candidates:
        thr, compact, cl = _shape(cand)
        probe = _lib.Params(params.tenure, min(params.iterations, probe_iterations), params.cap_mode,
                            params.lam, cl, thr, params.timeout_ns,
                            (params.flags & ~COMPACT_LAYOUT) | (COMPACT_LAYOUT if compact else 0))
        try:
            solve_batch(bp, probe, out=out)  # warm-up
        except _lib.AschedError as e:
            if e.status == E_TOO_LARGE and cl > 1:
                continue
            raise
        best = None
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            solve_batch(bp, probe, out=out)
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        times[(thr, compact, cl)] = best
    return min(times, key=times.get), times


def tuned_params(params: _lib.Params, choice) -> _lib.Params:
    """params with the launch shape an autotune_batch choice names."""
    thr, compact, cl = _shape(choice)
    return _lib.Params(params.tenure, params.iterations, params.cap_mode, params.lam, cl,
                       int(thr), params.timeout_ns,
                       (params.flags & ~COMPACT_LAYOUT) | (COMPACT_LAYOUT if compact else 0))


def solve_batch_static(bp: BatchProblem, params: _lib.Params, out: Optional[BatchOutput] = None,
                       stream: Optional[torch.cuda.Stream] = None) -> BatchOutput:
    """Queue asched_solve_batch_static: the same solve as solve_batch, for callers that
    cannot provide device scratch memory; the library's fixed per-device array serves as
    the work queue instead of bp.workspace. Calls that overlap on the GPU race on that
    array, so keep them on one stream."""
    if out is None:
        out = bp.alloc_output()
    s = stream if stream is not None else torch.cuda.current_stream(bp.device)
    res = out.struct()
    rc = _lib.load().asched_solve_batch_static(ctypes.byref(bp.struct), ctypes.byref(params),
                                               ctypes.byref(res), ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_solve_batch_static")
    return out


def capture_batch(bp: BatchProblem, params: _lib.Params, out: Optional[BatchOutput] = None):
    """Capture one asched_solve_batch (its ordering kernel and persistent launch) into a
    CUDA graph. Returns (graph, out); graph.replay() reruns the whole batch into `out`.
    The batch's inputs may be rewritten in place between replays (same sizes)."""
    if out is None:
        out = bp.alloc_output()
    s = torch.cuda.Stream(device=bp.device)
    s.wait_stream(torch.cuda.current_stream(bp.device))
    with torch.cuda.stream(s):
        solve_batch(bp, params, out=out, stream=s)  # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        solve_batch(bp, params, out=out, stream=s)
    return g, out


def sweep_params(max_sweeps: int, cap_mode: int = HARD, lam: int = 1000, tenure: int = 0,
                 accept_worse: bool = False, block_threads: int = 0, repair: bool = False) -> _lib.Params:
    """Parameters of asched_sweep_batch: iterations holds the most sweeps; repair turns on
    Algorithm 1's repair sweep."""
    flags = (SWEEP_ACCEPT_WORSE if accept_worse else 0) | (SWEEP_REPAIR if repair else 0)
    return _lib.Params(int(tenure), int(max_sweeps), int(cap_mode), int(lam), 0, int(block_threads), 0,
                       flags)


@dataclasses.dataclass
class SweepTrace:
    move: torch.Tensor  # uint32 ids stored as int32, [B][capacity]
    z: torch.Tensor  # int32 [B][capacity]
    capacity: int

    def struct(self):
        return _lib.SweepTrace(_ptr(self.move), _ptr(self.z), int(self.capacity))


def sweep_orders_tensors(bp: BatchProblem, orders):
    """Pack per-instance (vehicle_order, mission_rank) pairs (numpy arrays, either may be
    None for the default) into the batch's concatenated device layout."""
    vo = np.concatenate([np.arange(int(bp.h_veh_off[b + 1] - bp.h_veh_off[b])) if o[0] is None else o[0]
                         for b, o in enumerate(orders)]).astype(np.int32)
    mr = np.concatenate([np.arange(int(bp.h_mis_off[b + 1] - bp.h_mis_off[b])) if o[1] is None else o[1]
                         for b, o in enumerate(orders)] or [np.zeros(0)]).astype(np.int32)
    t = lambda a: torch.from_numpy(a if a.size else np.zeros(1, np.int32)).to(bp.device)  # noqa: E731
    return t(vo), t(mr)


def sweep_batch(bp: BatchProblem, algorithm: int, params: _lib.Params, out: Optional[BatchOutput] = None,
                trace_capacity: int = 0, stream: Optional[torch.cuda.Stream] = None, orders=None):
    """Queue asched_sweep_batch: Algorithm 2 (SWEEP_NEIGHBOURHOOD) or the per-mission sweep
    of Algorithm 3 (SWEEP_TABU) on every instance. orders: None (index and route order),
    a pair of device tensors from sweep_orders_tensors, or a list of per-instance
    (vehicle_order, mission_rank). Returns (out, trace or None)."""
    if out is None:
        out = bp.alloc_output()
    trace = None
    if trace_capacity > 0:
        n = max(bp.B, 1) * int(trace_capacity)
        trace = SweepTrace(torch.zeros(n, dtype=torch.int32, device=bp.device),
                           torch.zeros(n, dtype=torch.int32, device=bp.device), int(trace_capacity))
    ords = None
    if orders is not None:
        vo, mr = orders if isinstance(orders, tuple) else sweep_orders_tensors(bp, orders)
        ords = _lib.SweepOrders(_ptr(vo), _ptr(mr))
        bp._keep_orders = (vo, mr)  # the launch reads them until the stream gets there
    s = stream if stream is not None else torch.cuda.current_stream(bp.device)
    res = out.struct()
    tr = trace.struct() if trace is not None else None
    rc = _lib.load().asched_sweep_batch(ctypes.byref(bp.struct), int(algorithm), ctypes.byref(params),
                                        ctypes.byref(ords) if ords is not None else None,
                                        ctypes.byref(res), ctypes.byref(tr) if tr is not None else None,
                                        ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_sweep_batch")
    return out, trace


METRIC_EUCLIDEAN, METRIC_HAVERSINE = _lib.METRIC_EUCLIDEAN, _lib.METRIC_HAVERSINE


def travel_into_batch(bp: BatchProblem, coords: torch.Tensor, speeds_kmh, metric: int = METRIC_EUCLIDEAN,
                      radius_km: float = 0.0, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Queue asched_travel_matrix: rebuild every instance's travel matrix in bp.travel from
    coords (device float64 [total locations, 2], instance b's rows at bp.h_loc_off[b]).
    Returns the device status word (ASCHED_OK, or E_INVALID for a non-finite coordinate
    or a time beyond int32)."""
    if coords.dtype != torch.float64 or tuple(coords.shape) != (int(bp.h_loc_off[-1]), 2):
        raise ValueError("coords must be a float64 [total locations, 2] tensor")
    coords = coords.to(bp.device).contiguous()
    sp = [float(x) for x in speeds_kmh]
    if len(sp) != bp.n_types:
        raise ValueError("one speed per travel layer")
    status = torch.zeros(1, dtype=torch.int32, device=bp.device)
    hp = ctypes.c_void_p(bp.h_loc_off.ctypes.data)
    spec = _lib.TravelSpec(bp.B, hp, _ptr(bp.loc_off), _ptr(bp.travel_off), _ptr(coords), bp.n_types,
                           (ctypes.c_double * 2)(*(sp + [1.0])[:2]), int(metric), float(radius_km))
    s = stream if stream is not None else torch.cuda.current_stream(bp.device)
    rc = _lib.load().asched_travel_matrix(ctypes.byref(spec), _ptr(bp.travel), _ptr(status),
                                          ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_travel_matrix")
    bp._keep_coords = coords  # the launch reads it until the stream gets there
    return status


def travel_matrix(coords, speeds_kmh, metric: int = METRIC_EUCLIDEAN, radius_km: float = 0.0,
                  device="cuda") -> torch.Tensor:
    """One instance's [n_types, L, L] int32 travel minutes built on the device from
    coords [L, 2] (see asched_travel_matrix)."""
    c = torch.as_tensor(np.ascontiguousarray(coords, dtype=np.float64)).to(device)
    L, nt = int(c.shape[0]), len(speeds_kmh)
    dev = torch.device(device)
    h_loc = np.array([0, L], dtype=np.int32)
    loc = torch.from_numpy(h_loc).to(dev)
    toff = torch.zeros(1, dtype=torch.int64, device=dev)
    out = torch.empty((nt, L, L), dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    sp = [float(x) for x in speeds_kmh]
    spec = _lib.TravelSpec(1, ctypes.c_void_p(h_loc.ctypes.data), _ptr(loc), _ptr(toff), _ptr(c), nt,
                           (ctypes.c_double * 2)(*(sp + [1.0])[:2]), int(metric), float(radius_km))
    s = torch.cuda.current_stream(dev)
    _lib.check(_lib.load().asched_travel_matrix(ctypes.byref(spec), _ptr(out), _ptr(status),
                                                ctypes.c_void_p(s.cuda_stream)), "asched_travel_matrix")
    s.synchronize()
    if int(status.item()) != OK:
        raise AschedError(int(status.item()), "asched_travel_matrix (device)")
    return out


# --------------------------------------------------------------- roofline probes --

def measure_sm_peaks(device="cuda", iters: int = 4000, repeats: int = 3):
    """Per-SM rates of the roofline probes (asched_probe_sm_peak): int32 operations (add /
    xor / min and add / xor mixes), conflict-free shared-memory words and randomly gathered shared-memory words per SM
    clock, each the median over SMs of (work of the SM's CTAs) / (cycles from the SM's
    first start to its last end), best of `repeats` launches. Also the SM count."""
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cap = 32 * sms
    rec = torch.zeros(3 * cap, dtype=torch.int64, device=dev)
    sink = torch.zeros(cap, dtype=torch.int32, device=dev)
    work = {_lib.PROBE_INT32: _lib.PROBE_INT32_OPS_PER_STEP,
            _lib.PROBE_INT32_ADD_XOR: _lib.PROBE_INT32_ADD_XOR_OPS_PER_STEP,
            _lib.PROBE_LDS: _lib.PROBE_LDS_LOADS_PER_STEP,
            _lib.PROBE_LDS_GATHER: _lib.PROBE_LDS_LOADS_PER_STEP}
    out = {"sms": sms}
    names = {_lib.PROBE_INT32: "int32_ops_per_clk_sm", _lib.PROBE_INT32_ADD_XOR: "int32_add_xor_ops_per_clk_sm",
             _lib.PROBE_LDS: "lds_words_per_clk_sm", _lib.PROBE_LDS_GATHER: "lds_gather_words_per_clk_sm"}
    s = torch.cuda.current_stream(dev)
    for kind, per_step in work.items():
        best = 0.0
        for _ in range(repeats + 1):  # the first launch is a warm-up
            ctas, threads = ctypes.c_int32(0), ctypes.c_int32(0)
            _lib.check(_lib.load().asched_probe_sm_peak(int(kind), int(iters), _ptr(rec), cap, _ptr(sink),
                                                        ctypes.byref(ctas), ctypes.byref(threads),
                                                        ctypes.c_void_p(s.cuda_stream)), "asched_probe_sm_peak")
            s.synchronize()
            r = rec[: 3 * ctas.value].view(-1, 3).cpu().numpy()
            rates = []
            for sm in np.unique(r[:, 0]):
                rows = r[r[:, 0] == sm]
                span = int(rows[:, 2].max() - rows[:, 1].min())
                if span > 0:
                    rates.append(len(rows) * threads.value * iters * per_step / span)
            best = max(best, float(np.median(rates)))
        out[names[kind]] = best
    return out
