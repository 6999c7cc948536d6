"""oat_backproject_noalloc: the backprojection for callers that cannot allocate device memory
when they call it.  Its scratch is an array in static device memory, so it must give the same
result as oat_backproject, call after call (the array keeps the previous call's contents and
each call must clear what it needs), and refuse volumes larger than the array."""
import ctypes

import numpy as np
import pytest

from paper_1304_2017_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1304_2017_gb300 import oat
    fn = oat.lib.oat_backproject_noalloc
    fn.argtypes = [ctypes.c_void_p] * 4
    fn.restype = ctypes.c_int
    return torch, oat, fn


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_backproject_twice(env):
    torch, oat, fn = env
    geom = W.make_geometry((40, 36, 44), 0.25, 4, 6, 9.0, 160)
    plan = oat.Plan(geom)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (31, 32):   # two calls in a row, different data
        y = torch.from_numpy(W.random_data(geom, seed=seed)).cuda()
        ref = plan.backproject(y)
        out = torch.full(plan.vol_shape, float("nan"), device="cuda")
        rc = fn(plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == oat.OAT_OK, oat.oat_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64)
        assert np.isfinite(o).all()
        assert _rel(o, r) <= TOL
    plan.close()


def _compare(env, plan, geom, y, calls=2):
    torch, oat, fn = env
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(calls):
        ref = plan.backproject(y)
        out = torch.full(plan.vol_shape, float("nan"), device="cuda")
        rc = fn(plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == oat.OAT_OK, oat.oat_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64)
        assert np.isfinite(o).all()
        assert _rel(o, r) <= TOL


def test_noalloc_at_the_voxel_limit(env):
    """128^3 = 2^21 voxels, exactly the size of the static array."""
    torch, oat, fn = env
    geom = W.make_geometry(128, 0.1, 2, 2, 20.0, 64)
    assert geom.n_voxels == 1 << 21
    plan = oat.Plan(geom)
    _compare(env, plan, geom, torch.from_numpy(W.random_data(geom, seed=33)).cuda())
    plan.close()


@pytest.mark.parametrize("variant", ["f16", "bf16", "eir", "exact_area"])
def test_noalloc_variants(env, variant):
    """FP16 / BF16 stored data, a transducer response (H^e^T first) and exact strip-area weights."""
    import dataclasses
    torch, oat, fn = env
    geom = W.make_geometry((24, 20, 28), 0.25, 3, 5, 9.0, 120)
    if variant == "exact_area":
        geom = dataclasses.replace(geom, lattice_weights=1)
    dtype = {"f16": oat.OAT_F16, "bf16": oat.OAT_BF16}.get(variant, oat.OAT_F32)
    plan = oat.Plan(geom, data_dtype=dtype)
    if variant == "eir":
        plan.set_eir(*W.eir_taps(kind="gaussian"))
    y = torch.from_numpy(W.random_data(geom, seed=34)).cuda().to(plan.torch_data_dtype)
    _compare(env, plan, geom, y)
    plan.close()


def test_noalloc_rejects_volume_over_limit(env):
    torch, oat, fn = env
    geom = W.make_geometry(129, 0.1, 1, 1, 20.0, 8)   # 129^3 > 2^21 voxels
    plan = oat.Plan(geom)
    y = torch.zeros(plan.data_shape, device="cuda")
    out = torch.zeros(plan.vol_shape, device="cuda")
    rc = fn(plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == oat.OAT_ERR_INVALID_ARG
    assert "static scratch" in oat.oat_last_error()
    plan.close()
