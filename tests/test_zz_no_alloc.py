"""asched_solve_batch_static, the batch solve for callers that cannot allocate device
memory (it uses the library's fixed per-device scratch array instead of a workspace),
must give exactly what asched_solve_batch gives, call after call. Collected last on
purpose, so that a failure here cannot hide another test's result."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2002_11710_gb300 import _lib, api, gen

pytestmark = pytest.mark.gpu


def _batch(seed0, n):
    insts = []
    for k in range(n):
        s = seed0 + k
        insts.append(gen.random_instance(s, n_loc=8 + s % 7, n_vehicles=2 + s % 5,
                                         n_missions=5 + (7 * s) % 60, n_types=2,
                                         duty_cap=1200, max_minutes=120))
    return insts


def _static_call(bp, params):
    """asched_solve_batch_static through the C ABI (ctypes), on torch's current stream."""
    out = bp.alloc_output()
    res = out.struct()
    rc = _lib.load().asched_solve_batch_static(ctypes.byref(bp.struct), ctypes.byref(params),
                                               ctypes.byref(res),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == api.OK, _lib.status_string(rc)
    return out


def _assert_same(a, b):
    for k in ("route_off", "route", "flight", "overflow", "info"):
        np.testing.assert_array_equal(getattr(a, k).cpu().numpy(), getattr(b, k).cpu().numpy(), err_msg=k)


def test_static_batch_equals_workspace_batch_two_calls_in_a_row():
    params = api.make_params(5, 80, api.PENALTY, 1000)
    first = api.BatchProblem(_batch(500, 37))
    second = api.BatchProblem(_batch(900, 53))  # a different, larger batch right after
    s1 = _static_call(first, params)
    s2 = _static_call(second, params)
    w1 = api.solve_batch(first, params)
    w2 = api.solve_batch(second, params)
    torch.cuda.synchronize()
    assert (s1.info.view(-1, api.INFO_LEN)[:, api.INFO_STATUS] == 0).all()
    assert (s2.info.view(-1, api.INFO_LEN)[:, api.INFO_STATUS] == 0).all()
    _assert_same(s1, w1)
    _assert_same(s2, w2)


def test_static_batch_rejects_batches_over_the_fixed_size():
    too_many = _lib.Batch()
    too_many.n_instances = _lib.STATIC_BATCH_MAX + 1
    out = _lib.BatchResult()
    params = api.make_params(5, 10, api.PENALTY, 1000)
    rc = _lib.load().asched_solve_batch_static(ctypes.byref(too_many), ctypes.byref(params),
                                               ctypes.byref(out), None)
    assert rc == api.E_TOO_LARGE
