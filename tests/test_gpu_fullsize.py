"""Parity at full size, in the launch configuration the benchmark times.

256^3 grid, 128 x 180 transducers on 65 mm, K = 1536 (FP32 data), and the sparse-view
128 x 60 scanner with FP16 / BF16 data storage.  The GPU runs H and H^T on the whole plan;
the FP64 oracle computes what it can in seconds:

- H: every row of a few sampled transducers (the oracle on the scanner restricted to them);
- H^T: the full volume for data that is zero except on the sampled transducers, which is the
  oracle's H^T on the restricted scanner;
- the adjoint identity with dense N(0,1) data over all transducers (FP64 inner products).
"""
import numpy as np
import pytest

import oracle
from paper_1304_2017_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
# one transducer per quadrant of the arc / view grid, plus the first and last
SAMPLE = {"c2": [0, 64 * 180 + 45, 100 * 180 + 137, 23039], "c5": [0, 31 * 60 + 17, 90 * 60 + 44, 7679]}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1304_2017_gb300 import oat
    return torch, oat


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check(env, name, dtype, store_tol):
    torch, oat = env
    geom = W.config(name)
    qs = SAMPLE[name]
    sub = geom.subset(qs)
    alpha = W.phantom(name, geom)
    plan = oat.Plan(geom, data_dtype=dtype)
    try:
        u = plan.project(torch.from_numpy(alpha).cuda())
        u_s = u[qs].float().cpu().numpy()
        errs = {"H": rel(u_s, oracle.H(sub, alpha))}
        # H^T of data living on the sampled transducers only
        y = torch.zeros(geom.data_shape, dtype=plan.torch_data_dtype, device="cuda")
        y_s = torch.from_numpy(W.random_data(sub, seed=31)).to(plan.torch_data_dtype)
        y[qs] = y_s.cuda()
        a = plan.backproject(y).cpu().numpy()
        errs["Ht"] = rel(a, oracle.Ht(sub, y_s.float().numpy()))
        # adjoint identity with dense data over the whole scanner
        yd = torch.from_numpy(W.random_data(geom, seed=32)).cuda().to(plan.torch_data_dtype)
        ad = plan.backproject(yd)
        lhs = float((u.double() * yd.double()).sum())
        rhs = float((torch.from_numpy(alpha).cuda().double() * ad.double()).sum())
        errs["adjoint"] = abs(lhs - rhs) / (float(u.double().norm()) * float(yd.double().norm()))
        torch.cuda.synchronize()
    finally:
        plan.close()
    print(name, dtype, errs)
    assert errs["H"] <= store_tol + TOL, errs
    assert errs["Ht"] <= TOL, errs
    assert errs["adjoint"] <= TOL, errs


def test_full_size_fp32(env):
    """256^3, 23,040 transducers, K = 1536, FP32 data."""
    check(env, "c2", 0, 0.0)


@pytest.mark.parametrize("dtype,store", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_full_size_half_storage(env, dtype, store):
    """256^3 sparse-view scanner with FP16 (dtype 1) / BF16 (dtype 2) data storage: the
    projector's error adds the storage rounding; the backprojector reads stored values exactly."""
    check(env, "c5", dtype, store)
