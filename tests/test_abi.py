"""The C ABI library builds, loads and exports every declared entry point; host-side
logic (sizes, validation of host data, status strings) works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_11710_gb300 import _lib, api, gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "asched.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asched_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    names = declared_functions()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_abi_version_and_status_strings():
    L = _lib.load()
    assert L.asched_abi_version() == _lib.ABI_VERSION == 2
    for rc in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(_lib.status_string(rc), str)
    assert _lib.status_string(0) == "ok"


def test_num_moves_closed_form():
    for M in range(0, 40, 7):
        for V in (1, 2, 5, 20):
            assert api.num_moves(M, V) == M * (M + V - 2) + M * (M - 1) // 2
    assert api.num_moves(100, 20) == 16750
    with pytest.raises(api.AschedError):
        api.num_moves(-1, 3)


def _params(**kw):
    return api.make_params(**{**dict(tenure=5, iterations=10, cap_mode=gen.PENALTY, lam=1000), **kw})


def test_check_instance_host_accepts_the_workloads():
    for inst in (gen.tiny(0), gen.paper_shaped(0), gen.large(0), gen.paper_model(1, 20)):
        assert api.check_instance_host(inst, _params()) == api.OK


def test_check_instance_host_rejects_bad_data():
    base = gen.random_instance(5, n_loc=6, n_vehicles=3, n_missions=8)

    def variant(**kw):
        return gen.Instance(**{**base.__dict__, **kw})

    p = base.pickup.copy(); p[2] = 6
    assert api.check_instance_host(variant(pickup=p), _params()) == api.E_INVALID
    d = base.delivery.copy(); d[1] = base.pickup[1]
    assert api.check_instance_host(variant(delivery=d), _params()) == api.E_INVALID
    t = base.travel.copy(); t[0, 1, 2] = -1
    assert api.check_instance_host(variant(travel=t), _params()) == api.E_INVALID
    vb = base.veh_base.copy(); vb[0] = -3
    assert api.check_instance_host(variant(veh_base=vb), _params()) == api.E_INVALID
    vt = base.veh_type.copy(); vt[0] = 1  # only one travel layer
    assert api.check_instance_host(variant(veh_type=vt), _params()) == api.E_INVALID
    h = np.zeros(8, np.int32); h[0] = 2
    assert api.check_instance_host(variant(heli_only=h), _params()) == api.E_INVALID
    big = variant(travel=base.travel * 100000)
    assert api.check_instance_host(big, _params()) == api.E_OVERFLOW_GUARD
    assert api.check_instance_host(big, _params(cap_mode=gen.HARD)) == api.OK


def test_check_instance_host_rejects_bad_params():
    inst = gen.tiny(0)
    assert api.check_instance_host(inst, _params(cap_mode=3)) == api.E_INVALID
    assert api.check_instance_host(inst, _params(tenure=-1)) == api.E_INVALID
    assert api.check_instance_host(inst, _params(cluster_size=5)) == api.E_INVALID
    assert api.check_instance_host(inst, _params(block_threads=100)) == api.E_INVALID
    assert api.check_instance_host(inst, _params(block_threads=1024)) == api.E_INVALID
    assert api.check_instance_host(inst, _params(cluster_size=16, block_threads=64)) == api.OK
    assert api.check_instance_host(inst, _params(compact=True)) == api.OK
    p = _params()
    p.flags = 8
    assert api.check_instance_host(inst, p) == api.E_INVALID


def test_plan_without_a_device_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    inst = gen.tiny(0)
    s, keep = api.host_struct(inst)
    out = _lib.Plan()
    rc = _lib.load().asched_plan(ctypes.byref(s), ctypes.byref(_params()), ctypes.byref(out))
    assert rc == api.E_CUDA


def test_validate_and_workspace_entry_points_host_paths():
    """asched_validate is the host validation under the interface's name (no GPU needed).
    asched_workspace_bytes rejects bad arguments before it asks the device anything; with
    no device it reports the CUDA error, on a GPU the bytes of the plan's key slots."""
    L = _lib.load()
    base = gen.random_instance(5, n_loc=6, n_vehicles=3, n_missions=8)
    bad = gen.Instance(**{**base.__dict__, "pickup": np.where(np.arange(8) == 2, 6, base.pickup)})
    for inst in (base, gen.paper_shaped(0), bad):
        s, keep = api.host_struct(inst)
        p = _params()
        assert L.asched_validate(ctypes.byref(s), ctypes.byref(p)) == api.check_instance_host(inst, p)
    s, keep = api.host_struct(gen.paper_shaped(0))
    n = ctypes.c_size_t(123)
    import torch
    rc = L.asched_workspace_bytes(ctypes.byref(s), ctypes.byref(_params()), ctypes.byref(n))
    if torch.cuda.is_available():
        assert rc == api.OK and n.value == 0  # one cluster: all state on chip
    else:
        assert rc == api.E_CUDA
    assert L.asched_workspace_bytes(ctypes.byref(s), ctypes.byref(_params(grid_clusters=-1)),
                                    ctypes.byref(n)) == api.E_INVALID
    assert L.asched_workspace_bytes(ctypes.byref(s), ctypes.byref(_params(cap_mode=9)),
                                    ctypes.byref(n)) == api.E_INVALID
    assert L.asched_workspace_bytes(ctypes.byref(s), ctypes.byref(_params()), None) == api.E_INVALID


def test_binding_constants_match_the_header():
    """Every integer #define ASCHED_<NAME> of include/asched.h that the binding mirrors
    (as _lib.<NAME>) has the same value there (status codes in parentheses included)."""
    import re

    from paper_2002_11710_gb300 import _lib

    text = open(os.path.join(ROOT, "include", "asched.h")).read()
    checked = 0
    for name, val in re.findall(r"#define ASCHED_([A-Z0-9_]+)\s+\(?(-?(?:0x[0-9A-Fa-f]+|\d+))u?\)?", text):
        if hasattr(_lib, name):
            assert getattr(_lib, name) == int(val, 0), name
            checked += 1
    assert checked >= 40
