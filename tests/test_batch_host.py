"""Batch packing (host side, no GPU): concatenated arrays and offsets."""
import numpy as np
import pytest

from paper_2002_11710_gb300 import api, gen


def test_pack_offsets_and_contents():
    insts = [gen.random_instance(s, n_loc=5 + s, n_vehicles=1 + s % 3, n_missions=3 * s,
                                 n_types=2, heli_only_frac=0.3 if s % 2 else 0.0)
             for s in range(5)]
    bp = api.BatchProblem(insts, device="cpu")
    assert bp.B == 5 and bp.n_types == 2
    np.testing.assert_array_equal(bp.h_loc_off, np.cumsum([0] + [5 + s for s in range(5)]))
    np.testing.assert_array_equal(bp.h_mis_off, np.cumsum([0] + [3 * s for s in range(5)]))
    for b, inst in enumerate(insts):
        vo, mo = bp.h_veh_off[b], bp.h_mis_off[b]
        L = inst.n_loc
        t0 = int(bp.h_travel_off[b])
        np.testing.assert_array_equal(bp.travel[t0:t0 + 2 * L * L].numpy(), inst.travel.reshape(-1))
        np.testing.assert_array_equal(bp.veh_base[vo:vo + inst.n_vehicles].numpy(), inst.veh_base)
        np.testing.assert_array_equal(bp.pickup[mo:mo + inst.n_missions].numpy(), inst.pickup)
        h = inst.heli_only if inst.heli_only is not None else np.zeros(inst.n_missions)
        np.testing.assert_array_equal(bp.heli_only[mo:mo + inst.n_missions].numpy(), h)
    out = bp.alloc_output()
    assert out.route_off.numel() == bp.h_veh_off[-1] + bp.B
    assert out.info.numel() == 5 * api.INFO_LEN


def test_pack_rejects_mixed_layers_and_deadlines():
    a = gen.random_instance(1, n_loc=5, n_vehicles=2, n_missions=4, n_types=1)
    b = gen.random_instance(2, n_loc=5, n_vehicles=2, n_missions=4, n_types=2)
    with pytest.raises(ValueError):
        api.BatchProblem([a, b], device="cpu")
    c = gen.random_instance(3, n_loc=5, n_vehicles=2, n_missions=4, deadlines=True)
    with pytest.raises(ValueError):
        api.BatchProblem([a, c], device="cpu")


def test_workload_batches_pack():
    for insts in ([gen.batched_member(i) for i in range(64)],
                  [gen.random_instance(300 + s, n_loc=8, n_vehicles=3, n_missions=10, n_types=2)
                   for s in range(3)] + [gen.random_instance(9, n_loc=30, n_vehicles=6, n_missions=90,
                                                             n_types=2)]):
        bp = api.BatchProblem(insts, device="cpu")
        assert bp.B == len(insts)


def test_sweep_host_argument_errors_need_no_gpu():
    """asched_sweep_batch rejects bad arguments on the host before any CUDA call."""
    import ctypes

    from paper_2002_11710_gb300 import _lib
    insts = [gen.random_instance(s, n_loc=6, n_vehicles=2, n_missions=4) for s in range(3)]
    bp = api.BatchProblem(insts, device="cpu")
    out = bp.alloc_output().struct()
    L = _lib.load()

    def call(alg, p, trace=None):
        return L.asched_sweep_batch(ctypes.byref(bp.struct), alg, ctypes.byref(p), None, ctypes.byref(out),
                                    ctypes.byref(trace) if trace is not None else None, None)

    assert call(9, api.sweep_params(5)) == api.E_INVALID
    assert call(api.SWEEP_NEIGHBOURHOOD, api.sweep_params(5, accept_worse=True)) == api.E_INVALID
    assert call(api.SWEEP_TABU, api.sweep_params(5, block_threads=48)) == api.E_INVALID
    assert call(api.SWEEP_TABU, api.sweep_params(5, block_threads=1024)) == api.E_INVALID
    assert call(api.SWEEP_TABU, api.sweep_params(-1)) == api.E_INVALID
    assert call(api.SWEEP_TABU, api.sweep_params(5, cap_mode=7)) == api.E_INVALID
    p = api.sweep_params(5)
    p.cluster_size = 2
    assert call(api.SWEEP_TABU, p) == api.E_INVALID
    p = api.sweep_params(5)
    p.flags = api.COMPACT_LAYOUT
    assert call(api.SWEEP_TABU, p) == api.E_INVALID
    assert call(api.SWEEP_TABU, api.sweep_params(5), _lib.SweepTrace(None, None, -1)) == api.E_INVALID
    empty = api.BatchProblem([], device="cpu")
    assert L.asched_sweep_batch(ctypes.byref(empty.struct), api.SWEEP_TABU, ctypes.byref(api.sweep_params(5)),
                                None, ctypes.byref(empty.alloc_output().struct()), None, None) == api.OK


def test_travel_host_argument_errors_need_no_gpu():
    """asched_travel_matrix rejects bad specs on the host before any CUDA call (status
    NULL, so nothing touches a device)."""
    import ctypes

    from paper_2002_11710_gb300 import _lib
    L = _lib.load()
    off = np.array([0, 3, 7], dtype=np.int32)
    fake = ctypes.c_void_p(16)  # device pointers the host never dereferences
    travel = ctypes.c_void_p(64)

    def spec(**kw):
        f = dict(n=2, h=off, nt=2, speeds=(300.0, 500.0), metric=api.METRIC_EUCLIDEAN, radius=0.0)
        f.update(kw)
        h = f["h"]
        return _lib.TravelSpec(f["n"], ctypes.c_void_p(h.ctypes.data) if h is not None else None, fake, fake, fake,
                               f["nt"], (ctypes.c_double * 2)(*f["speeds"]), f["metric"], f["radius"])

    def call(s, out=travel):
        return L.asched_travel_matrix(ctypes.byref(s) if s is not None else None, out, None, None)

    assert call(None) == api.E_INVALID
    assert call(spec(), out=None) == api.E_INVALID
    for kw in (dict(n=-1), dict(nt=0), dict(nt=3), dict(metric=7), dict(speeds=(0.0, 500.0)),
               dict(speeds=(300.0, -1.0)), dict(speeds=(float("inf"), 500.0)), dict(speeds=(float("nan"), 500.0)),
               dict(metric=api.METRIC_HAVERSINE, radius=-1.0),
               dict(metric=api.METRIC_HAVERSINE, radius=float("inf")), dict(h=None),
               dict(h=np.array([1, 3, 7], dtype=np.int32)), dict(h=np.array([0, 3, 3], dtype=np.int32))):
        assert call(spec(**kw)) == api.E_INVALID, kw
    assert call(spec(n=0)) == api.OK  # nothing to build
