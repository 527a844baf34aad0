"""ctypes view of the C ABI in include/asched.h (argument marshalling only).

The library is loaded from the package's own _build/ directory. There is no
fallback: if it is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

OK = 0
E_INVALID = -1
E_TOO_LARGE = -2
E_OVERFLOW_GUARD = -3
E_INFEASIBLE_INIT = -4
E_TIMEOUT = -5
E_CUDA = -6

STATIC_BATCH_MAX = 16384  # ASCHED_STATIC_BATCH_MAX
ABI_VERSION = 2  # ASCHED_ABI_VERSION

HARD = 0
PENALTY = 1
COMPACT_LAYOUT = 1  # asched_params.flags bits
TEST_WITHHOLD_KEY = 2
PLAIN_LAUNCH = 4

FLAG_FEASIBLE, FLAG_TABU, FLAG_ASPIRATION, FLAG_ADMISSIBLE = 1, 2, 4, 8
SWAP_BIT = 0x80000000
NULL_MOVE = 0xFFFFFFFF

INFO_STATUS, INFO_Z_BEST, INFO_BEST_IT, INFO_Z_INIT, INFO_Z_FINAL, INFO_ITERS = range(6)
INFO_LEN = 8

P = ctypes.c_void_p


class Instance(ctypes.Structure):
    _fields_ = [("n_loc", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("n_vehicles", ctypes.c_int32), ("n_missions", ctypes.c_int32),
                ("travel", P), ("veh_base", P), ("veh_type", P), ("pickup", P),
                ("delivery", P), ("heli_only", P), ("deadline", P),
                ("duty_cap", ctypes.c_int32), ("horizon", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("tenure", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("cap_mode", ctypes.c_int32), ("lam", ctypes.c_int32),
                ("cluster_size", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("timeout_ns", ctypes.c_int64), ("flags", ctypes.c_uint32),
                ("grid_clusters", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("moves_per_iteration", ctypes.c_int64),
                ("grid_clusters", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("route_off", P), ("route", P), ("flight", P), ("overflow", P), ("info", P),
                ("traj_move", P), ("traj_z", P)]


class Server(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("ring_len", ctypes.c_int32),
                ("max_loc", ctypes.c_int32), ("max_vehicles", ctypes.c_int32),
                ("max_missions", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("has_deadlines", ctypes.c_int32), ("slot_data", P), ("slot_out", P),
                ("ring", P), ("control", P), ("done", P)]


SLOT_HEADER = 16
CTRL_PUBLISHED, CTRL_CLAIMED, CTRL_STOP, CTRL_SERVED, CTRL_IDLE_EXITS, CTRL_STARTED = 0, 1, 2, 3, 4, 5
CTRL_LEN = 8


class Batch(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("h_loc_off", P), ("h_veh_off", P), ("h_mis_off", P),
                ("loc_off", P), ("veh_off", P), ("mis_off", P), ("travel_off", P),
                ("travel", P), ("veh_base", P), ("veh_type", P), ("pickup", P), ("delivery", P),
                ("heli_only", P), ("deadline", P), ("duty_cap", P), ("horizon", P)]


class BatchResult(ctypes.Structure):
    _fields_ = [("route_off", P), ("route", P), ("flight", P), ("overflow", P), ("info", P)]


class SweepOrders(ctypes.Structure):
    _fields_ = [("vehicle_order", P), ("mission_rank", P)]


class SweepTrace(ctypes.Structure):
    _fields_ = [("move", P), ("z", P), ("capacity", ctypes.c_int32)]


class TravelSpec(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("h_loc_off", P), ("loc_off", P),
                ("travel_off", P), ("coords", P), ("n_types", ctypes.c_int32),
                ("speed_kmh", ctypes.c_double * 2), ("metric", ctypes.c_int32),
                ("radius_km", ctypes.c_double)]


METRIC_EUCLIDEAN, METRIC_HAVERSINE = 0, 1

SWEEP_NEIGHBOURHOOD = 2  # Algorithm 2
SWEEP_TABU = 3  # Algorithm 3 as printed
SWEEP_ACCEPT_WORSE = 4  # asched_params.flags bits for the sweeps
SWEEP_REPAIR = 8
INFO_MOVES, INFO_STEPS = 6, 7

PROBE_INT32, PROBE_LDS, PROBE_LDS_GATHER, PROBE_INT32_ADD_XOR = 0, 1, 2, 3
PROBE_INT32_OPS_PER_STEP, PROBE_LDS_LOADS_PER_STEP, PROBE_INT32_ADD_XOR_OPS_PER_STEP = 96, 16, 64


# Every entry point of include/asched.h with its ctypes signature.
SIGNATURES = {
    "asched_abi_version": (ctypes.c_int, []),
    "asched_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "asched_num_moves": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P]),
    "asched_check_instance_host": (ctypes.c_int, [P, P]),
    "asched_plan": (ctypes.c_int, [P, P, P]),
    "asched_solve": (ctypes.c_int, [P, P, P, P, P, P]),
    "asched_eval_neighbourhood": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int32, ctypes.c_int32,
                                                 P, P, P, P, P, P]),
    "asched_batch_workspace_bytes": (ctypes.c_int, [ctypes.c_int32, P]),
    "asched_solve_batch": (ctypes.c_int, [P, P, P, P, ctypes.c_size_t, P]),
    "asched_solve_batch_static": (ctypes.c_int, [P, P, P, P]),
    "asched_server_sizes": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, P, P]),
    "asched_serve": (ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_int32, P]),
    "asched_sweep_batch": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P, P]),
    "asched_travel_matrix": (ctypes.c_int, [P, P, P, P]),
    "asched_validate": (ctypes.c_int, [P, P]),
    "asched_workspace_bytes": (ctypes.c_int, [P, P, P]),
    "asched_greedy_init": (ctypes.c_int, [P, P, P, P, P, P]),
    "asched_tabu_solve": (ctypes.c_int, [P, P, P, P, P, P, ctypes.c_size_t, P]),
    "asched_probe_sm_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the in-tree library (building it first if it is absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library not built: {path}")
                _build.build()
            L = ctypes.CDLL(path)
            if L.asched_abi_version() != ABI_VERSION:
                raise RuntimeError(f"{path}: ABI version {L.asched_abi_version()}, expected {ABI_VERSION}")
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(rc: int) -> str:
    return load().asched_status_string(int(rc)).decode()


class AschedError(RuntimeError):
    def __init__(self, rc: int, where: str):
        super().__init__(f"{where}: {status_string(rc)} ({rc})")
        self.status = rc


def check(rc: int, where: str) -> None:
    if rc != OK:
        raise AschedError(rc, where)
