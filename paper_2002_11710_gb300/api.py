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
from ._lib import (E_CUDA, E_INFEASIBLE_INIT, E_INVALID, E_OVERFLOW_GUARD, E_TIMEOUT,  # noqa: F401
                   E_TOO_LARGE, FLAG_ADMISSIBLE, FLAG_ASPIRATION, FLAG_FEASIBLE, FLAG_TABU, HARD,
                   INFO_BEST_IT, INFO_ITERS, INFO_LEN, INFO_STATUS, INFO_Z_BEST, INFO_Z_FINAL,
                   INFO_Z_INIT, NULL_MOVE, OK, PENALTY, SWAP_BIT, AschedError)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def num_moves(n_missions: int, n_vehicles: int) -> int:
    out = ctypes.c_int64(0)
    _lib.check(_lib.load().asched_num_moves(int(n_missions), int(n_vehicles), ctypes.byref(out)),
               "asched_num_moves")
    return int(out.value)


def make_params(tenure: int, iterations: int, cap_mode: int = HARD, lam: int = 1000,
                cluster_size: int = 0, block_threads: int = 0, timeout_ns: int = 0) -> _lib.Params:
    return _lib.Params(int(tenure), int(iterations), int(cap_mode), int(lam), int(cluster_size),
                       int(block_threads), int(timeout_ns), 0)


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
          trajectory: bool = False, stream: Optional[torch.cuda.Stream] = None) -> SolveOutput:
    """Queue one Tabu search (asched_solve) on `stream` (default: torch's current stream).

    init: None (greedy start, Algorithm 1) or (route_off, route) device int32 tensors.
    Returns the output tensors; read them after synchronising the stream.
    """
    if out is None:
        out = alloc_output(dp, params.iterations, trajectory)
    s = stream if stream is not None else torch.cuda.current_stream(dp.device)
    res = out.struct()
    ioff, iroute = (None, None) if init is None else (_ptr(init[0]), _ptr(init[1]))
    rc = _lib.load().asched_solve(ctypes.byref(dp.struct), ctypes.byref(params), ioff, iroute,
                                  ctypes.byref(res), ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "asched_solve")
    return out


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
