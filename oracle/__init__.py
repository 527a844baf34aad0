"""Plain CPU oracle for the search methods of arXiv 2002.11710 (Algorithms 1, 2 and 3).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU baseline leg of
``bench.py`` are the only callers. The product path (the CUDA library and its
binding) never imports this package, and this package imports nothing from it.

The arithmetic lives in ``asched_oracle.c`` (plain C, full recompute of every
candidate schedule, 64-bit costs); this module compiles it with gcc on first use and
wraps it with ctypes. The independent moves of a neighbourhood are evaluated on OpenMP
threads and the chosen move is picked afterwards in canonical order, so results do not
depend on the thread count. Its readings of the paper are listed at the top of the C
file.

Pinned by ``tests/test_oracle_pins.py`` against brute force over every schedule of
tiny instances, the ILP's arc form of the objective and constraints (Section 3),
closed forms, an independent characterisation of the neighbourhood, and
hand-worked instances under ``tests/golden/``. The tie-break and tabu bookkeeping
of the trajectory are readings (R5-R7) that the paper does not print: the whole
trajectory's parity is "parity unpinned" beyond those pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "asched_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

FEASIBLE, TABU, ASPIRATION, ADMISSIBLE = 1, 2, 4, 8
SWAP_BIT = 0x80000000
NULL_MOVE = 0xFFFFFFFF
OK, E_INVALID, E_INFEASIBLE_INIT = 0, -1, -4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc -O2 -fopenmp)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class _Inst(ctypes.Structure):
    _fields_ = [
        ("n_loc", ctypes.c_int32), ("n_types", ctypes.c_int32),
        ("n_vehicles", ctypes.c_int32), ("n_missions", ctypes.c_int32),
        ("travel", ctypes.c_void_p), ("veh_base", ctypes.c_void_p),
        ("veh_type", ctypes.c_void_p), ("pickup", ctypes.c_void_p),
        ("delivery", ctypes.c_void_p), ("heli_only", ctypes.c_void_p),
        ("deadline", ctypes.c_void_p),
        ("duty_cap", ctypes.c_int32), ("horizon", ctypes.c_int32),
        ("cap_mode", ctypes.c_int32), ("lam", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.orc_num_moves.restype = ctypes.c_int64
            L.orc_num_moves.argtypes = [ctypes.c_int32, ctypes.c_int32]
            L.orc_cost.restype = ctypes.c_int64
            L.orc_cost.argtypes = [P, P, P, P, P]
            L.orc_feasible.restype = ctypes.c_int32
            L.orc_feasible.argtypes = [P, P, P]
            L.orc_greedy_init.restype = ctypes.c_int32
            L.orc_greedy_init.argtypes = [P, P, P]
            L.orc_eval_neighbourhood.restype = ctypes.c_int64
            L.orc_eval_neighbourhood.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int64,
                                                 P, P, P, P]
            L.orc_apply_tabu_move.restype = ctypes.c_int32
            L.orc_apply_tabu_move.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, P,
                                              ctypes.c_uint32]
            L.orc_tabu_search.restype = ctypes.c_int32
            L.orc_tabu_search.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P,
                                          P, P]
            L.orc_neighbourhood_search.restype = ctypes.c_int32
            L.orc_greedy_init_repair.restype = ctypes.c_int32
            L.orc_greedy_init_repair.argtypes = [P, P, P]
            L.orc_neighbourhood_search.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P,
                                                   P, P, P, P, P, ctypes.c_int64]
            L.orc_set_threads.restype = ctypes.c_int32
            L.orc_set_threads.argtypes = [ctypes.c_int32]
            L.orc_tabu_sweep.restype = ctypes.c_int32
            L.orc_tabu_sweep.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, P, P, P, P, P, P, P, P, P, P, ctypes.c_int64]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """An instance plus cap mode and penalty weight, held in C-compatible arrays."""

    def __init__(self, inst, cap_mode: int, lam: int = 1000):
        self.inst = inst
        self.cap_mode = int(cap_mode)
        self.lam = int(lam)
        c = np.ascontiguousarray
        self._keep = [c(inst.travel, dtype=np.int32), c(inst.veh_base, dtype=np.int32),
                      c(inst.veh_type, dtype=np.int32), c(inst.pickup, dtype=np.int32),
                      c(inst.delivery, dtype=np.int32),
                      None if inst.heli_only is None else c(inst.heli_only, dtype=np.int32),
                      None if inst.deadline is None else c(inst.deadline, dtype=np.int32)]
        t, vb, vt, p, d, h, w = self._keep
        self.M = int(p.shape[0])
        self.V = int(vb.shape[0])
        self._s = _Inst(int(t.shape[1]), int(t.shape[0]), self.V, self.M, _ptr(t), _ptr(vb),
                        _ptr(vt), _ptr(p), _ptr(d), _ptr(h), _ptr(w), int(inst.duty_cap),
                        int(inst.horizon), self.cap_mode, self.lam)

    @property
    def ref(self):
        return ctypes.byref(self._s)


def set_threads(n: int = 0) -> int:
    """Threads of the loop over moves in eval_neighbourhood / tabu_search (0: one per
    processor). Returns the count now in force. Results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def num_moves(M: int, V: int) -> int:
    return int(lib().orc_num_moves(M, V))


def cost(pb: Problem, off, route):
    """Objective and per-vehicle flight / overflow of a CSR schedule."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    route = np.ascontiguousarray(route, dtype=np.int32)
    fl = np.zeros(pb.V, dtype=np.int64)
    ov = np.zeros(pb.V, dtype=np.int64)
    z = lib().orc_cost(pb.ref, _ptr(off), _ptr(route), _ptr(fl), _ptr(ov))
    return int(z), fl, ov


def feasible(pb: Problem, off, route) -> bool:
    off = np.ascontiguousarray(off, dtype=np.int32)
    route = np.ascontiguousarray(route, dtype=np.int32)
    return bool(lib().orc_feasible(pb.ref, _ptr(off), _ptr(route)))


def greedy_init(pb: Problem, repair: bool = False):
    """Algorithm 1 (reading R8; with repair, R12). Returns (status, route_off, route)."""
    off = np.zeros(pb.V + 1, dtype=np.int32)
    route = np.zeros(max(pb.M, 1), dtype=np.int32)
    fn = lib().orc_greedy_init_repair if repair else lib().orc_greedy_init
    rc = fn(pb.ref, _ptr(off), _ptr(route))
    return int(rc), off, route[:pb.M]


def eval_neighbourhood(pb: Problem, off, route, tabu_until, it: int, z_best: int):
    """Every canonical move: (ids, delta, flags, chosen index or -1)."""
    off = np.ascontiguousarray(off, dtype=np.int32)
    route = np.ascontiguousarray(route, dtype=np.int32)
    tabu = np.ascontiguousarray(tabu_until, dtype=np.int32).reshape(-1)
    n = num_moves(pb.M, pb.V)
    delta = np.zeros(max(n, 1), dtype=np.int64)
    flags = np.zeros(max(n, 1), dtype=np.uint8)
    ids = np.zeros(max(n, 1), dtype=np.uint32)
    chosen = ctypes.c_int64(-1)
    got = lib().orc_eval_neighbourhood(pb.ref, _ptr(off), _ptr(route), _ptr(tabu), int(it),
                                       int(z_best), _ptr(delta), _ptr(flags), _ptr(ids),
                                       ctypes.addressof(chosen))
    if got < 0:
        raise RuntimeError(f"oracle eval_neighbourhood failed: {got}")
    return ids[:n], delta[:n], flags[:n], int(chosen.value)


def apply_tabu_move(pb: Problem, tenure: int, it: int, off, route, tabu_until, move_id: int):
    """Apply a move (or NULL_MOVE) in place on (off, route, tabu_until)."""
    rc = lib().orc_apply_tabu_move(pb.ref, int(tenure), int(it), _ptr(off), _ptr(route),
                                   _ptr(tabu_until), ctypes.c_uint32(int(move_id) & 0xFFFFFFFF))
    if rc != OK:
        raise RuntimeError(f"oracle apply_tabu_move failed: {rc}")


def tabu_search(pb: Problem, tenure: int, iterations: int, init=None):
    """Algorithm 3 (readings R5-R7). Returns a dict with status, best schedule, z_best,
    best_it, and the per-iteration trajectory (move ids, objectives)."""
    off = np.zeros(pb.V + 1, dtype=np.int32)
    route = np.zeros(max(pb.M, 1), dtype=np.int32)
    traj_move = np.zeros(max(iterations, 1), dtype=np.uint32)
    traj_z = np.zeros(max(iterations, 1), dtype=np.int64)
    zb = ctypes.c_int64(0)
    bi = ctypes.c_int32(0)
    if init is not None:
        ioff = np.ascontiguousarray(init[0], dtype=np.int32)
        iroute = np.ascontiguousarray(init[1], dtype=np.int32)
        ip = (_ptr(ioff), _ptr(iroute))
    else:
        ip = (None, None)
    rc = lib().orc_tabu_search(pb.ref, int(tenure), int(iterations), ip[0], ip[1], _ptr(off),
                               _ptr(route), ctypes.addressof(zb), ctypes.addressof(bi),
                               _ptr(traj_move), _ptr(traj_z))
    return {"status": int(rc), "route_off": off, "route": route[:pb.M], "z_best": int(zb.value),
            "best_it": int(bi.value), "traj_move": traj_move[:iterations],
            "traj_z": traj_z[:iterations]}


def _sweep(pb: Problem, fn, args, init, trace_cap, vorder, mrank):
    off = np.zeros(pb.V + 1, dtype=np.int32)
    route = np.zeros(max(pb.M, 1), dtype=np.int32)
    moves = np.zeros(max(trace_cap, 1), dtype=np.uint32)
    zs = np.zeros(max(trace_cap, 1), dtype=np.int64)
    zo = np.zeros(3, dtype=np.int64)
    counts = np.zeros(4, dtype=np.int32)
    if init is not None:
        ioff = np.ascontiguousarray(init[0], dtype=np.int32)
        iroute = np.ascontiguousarray(init[1], dtype=np.int32)
        ip = (_ptr(ioff), _ptr(iroute))
    else:
        ip = (None, None)
    vo = None if vorder is None else np.ascontiguousarray(vorder, dtype=np.int32)
    mr = None if mrank is None else np.ascontiguousarray(mrank, dtype=np.int32)
    rc = fn(pb.ref, *args, _ptr(vo), _ptr(mr), ip[0], ip[1], _ptr(off), _ptr(route), _ptr(zo),
            _ptr(counts), _ptr(moves), _ptr(zs), int(trace_cap))
    n = min(int(counts[2]), trace_cap)
    return {"status": int(rc), "route_off": off, "route": route[:pb.M], "z_best": int(zo[0]),
            "z_init": int(zo[1]), "z_final": int(zo[2]), "sweeps": int(counts[0]),
            "n_moves": int(counts[1]), "steps": int(counts[2]), "best_step": int(counts[3]),
            "trace_move": moves[:n], "trace_z": zs[:n]}


def neighbourhood_search(pb: Problem, max_sweeps: int, repair: bool = False, init=None,
                         trace_cap: int = 1 << 16, vorder=None, mrank=None):
    """Algorithm 2 (readings S1-S3, S5 in the C file) from Algorithm 1 (R8, or R12 with
    repair). One trace entry per mission step. vorder / mrank: the loop orders (S1)."""
    return _sweep(pb, lib().orc_neighbourhood_search, (int(max_sweeps), int(bool(repair))), init,
                  trace_cap, vorder, mrank)


def tabu_sweep(pb: Problem, tenure: int, max_sweeps: int, accept_worse: bool = False,
               repair: bool = False, init=None, trace_cap: int = 1 << 16, vorder=None, mrank=None):
    """Algorithm 3 as printed: per-mission sweep with a tabu list (readings S1, S2, S4 or,
    with accept_worse, S4b; S5)."""
    return _sweep(pb, lib().orc_tabu_sweep, (int(tenure), int(max_sweeps), int(bool(accept_worse)),
                                             int(bool(repair))), init, trace_cap, vorder, mrank)
