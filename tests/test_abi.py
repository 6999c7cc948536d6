"""The C-ABI library loads, exports every symbol include/oat.h declares, and rejects
invalid input on the host (no GPU work).  CPU only."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1304_2017_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|const char \*|void)\s*\*?\s*(oat_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def oat():
    import __graft_entry__ as ge
    from paper_1304_2017_gb300 import build as b
    b.build()
    del ge
    from paper_1304_2017_gb300 import oat as mod
    return mod


def test_exports_every_declared_symbol(oat):
    names = _declared()
    assert {"oat_plan_create", "oat_plan_destroy", "oat_project", "oat_backproject", "oat_plan_query",
            "oat_last_error"} <= names
    lib = ctypes.CDLL(oat.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert oat.oat_version() >= 10000


def _struct(oat, geom, **kw):
    s, pos = oat.make_geometry_struct(geom)
    for k, v in kw.items():
        setattr(s, k, v)
    return s, pos


@pytest.mark.parametrize("field,value,code", [
    ("nx", 0, -1), ("n_samples", 2, -1), ("spacing_mm", 0.0, -1), ("spacing_mm", float("nan"), -1),
    ("fs_mhz", -1.0, -1), ("c_mm_per_us", 0.0, -1), ("t_min_us", -0.5, -1), ("data_dtype", 7, -1),
    ("apply_d", 2, -1), ("support_radius_mm", 30.0, -2), ("t_min_us", 1000.0, -2),
    ("gruneisen", float("inf"), -1), ("lattice_weights", 2, -1), ("lattice_weights", -1, -1),
])
def test_invalid_geometry_rejected_on_host(oat, field, value, code):
    geom = W.make_geometry(8, 0.5, 2, 2, 10.0, 32)
    s, pos = _struct(oat, geom, **{field: value})
    h = ctypes.c_void_p(12345)
    rc = oat.lib.oat_plan_create(ctypes.byref(s), 0, ctypes.byref(h))
    assert rc == code, (rc, oat.oat_last_error())
    assert h.value is None
    assert oat.oat_last_error()


def test_non_finite_position_and_null_args(oat):
    geom = W.make_geometry(8, 0.5, 2, 2, 10.0, 32)
    geom.positions_mm[1, 2] = math.nan
    s, pos = _struct(oat, geom)
    h = ctypes.c_void_p()
    assert oat.lib.oat_plan_create(ctypes.byref(s), 0, ctypes.byref(h)) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_plan_create(None, 0, ctypes.byref(h)) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_project(None, None, None, None) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_backproject(None, None, None, None) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_plan_destroy(None) == oat.OAT_OK


def test_transducer_inside_support_sphere_rejected(oat):
    geom = W.make_geometry(8, 0.5, 2, 2, 10.0, 32)
    geom.positions_mm[0] = (0.1, 0.2, 0.3)
    s, pos = _struct(oat, geom)
    h = ctypes.c_void_p()
    assert oat.lib.oat_plan_create(ctypes.byref(s), 0, ctypes.byref(h)) == oat.OAT_ERR_GEOMETRY
    assert "support sphere" in oat.oat_last_error()


def test_valid_plan_without_gpu_fails_loudly(oat):
    """No CPU fallback: on a machine without a GPU a valid plan reports a CUDA error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    geom = W.make_geometry(8, 0.5, 2, 2, 10.0, 32)
    s, pos = _struct(oat, geom)
    h = ctypes.c_void_p()
    assert oat.lib.oat_plan_create(ctypes.byref(s), 0, ctypes.byref(h)) == oat.OAT_ERR_CUDA
    assert h.value is None


def _sph_create(oat, geom, n_freq, f0, df, eir=None):
    s, pos = _struct(oat, geom)
    h = ctypes.c_void_p(12345)
    e = None
    if eir is not None:
        e = np.ascontiguousarray(eir, dtype=np.float64)
    ptr = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if e is not None else None
    rc = oat.lib.oat_sph_create(ctypes.byref(s), n_freq, f0, df, ptr, 0, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("n_freq,f0,df", [(0, 0.1, 0.1), (4, 0.0, 0.1), (4, -1.0, 0.1), (4, 0.5, 0.0),
                                          (4, 0.5, -0.1), (4, math.nan, 0.1), (20000, 0.1, 0.1)])
def test_sph_bad_frequencies_rejected_on_host(oat, n_freq, f0, df):
    geom = W.make_geometry(6, 0.3, 1, 2, 5.0, 16)
    rc, h = _sph_create(oat, geom, n_freq, f0, df)
    assert rc == oat.OAT_ERR_INVALID_ARG, oat.oat_last_error()
    assert h.value is None


def test_sph_host_validation(oat):
    geom = W.make_geometry(6, 0.3, 1, 2, 5.0, 16, positions_mm=[[0.15, 0.15, 0.15], [5.0, 0, 0]])
    rc, _ = _sph_create(oat, geom, 4, 0.5, 0.1)                  # transducer 0 inside a voxel sphere
    assert rc == oat.OAT_ERR_INVALID_ARG and "inside a spherical voxel" in oat.oat_last_error()
    geom = W.make_geometry(6, 0.3, 1, 2, 5.0, 16)
    rc, _ = _sph_create(oat, geom, 3, 0.5, 0.1, eir=[1.0, 0.0, math.inf, 0.0, 1.0, 0.0])
    assert rc == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_sph_project(None, None, None, None) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_sph_backproject(None, None, None, None) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_sph_destroy(None) == oat.OAT_OK
    # no CPU fallback: a valid operator needs the GPU
    import torch
    if not torch.cuda.is_available():
        rc, h = _sph_create(oat, geom, 4, 0.5, 0.1)
        assert rc == oat.OAT_ERR_CUDA and h.value is None


def test_eir_and_fbp_null_args(oat):
    d = ctypes.POINTER(ctypes.c_double)()
    assert oat.lib.oat_plan_set_eir(None, d, 0, 0) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_plan_set_fbp_weights(None, d) == oat.OAT_ERR_INVALID_ARG
    assert oat.lib.oat_fbp(None, None, None, None) == oat.OAT_ERR_INVALID_ARG
