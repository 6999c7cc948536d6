"""GPU parity of the reconstruction layer: the FISTA-TV kernels against the FP64 reference
(oracle/recon.py), FISTA end to end, and the autograd wrapper's gradient against FP64 finite
differences of the oracle operator."""
import numpy as np
import pytest

import oracle
from oracle import recon
from paper_1304_2017_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1304_2017_gb300 import oat
    return torch, oat


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape", [(9, 13, 11), (1, 17, 20)])
@pytest.mark.parametrize("with_grad", [False, True])
def test_tv_prox_matches_reference(env, shape, with_grad):
    torch, oat = env
    rng = np.random.default_rng(4)
    z = (np.abs(rng.standard_normal(shape)) * (rng.random(shape) > 0.3)).astype(np.float32)
    g = rng.standard_normal(shape).astype(np.float32) if with_grad else None
    lam, iters, step = 0.08, 12, 0.3
    want = recon.tv_prox(z, lam, iters, g=g, step=step if with_grad else 0.0)
    zt = torch.from_numpy(z).cuda()
    gt = torch.from_numpy(g).cuda() if with_grad else None
    out = torch.empty_like(zt)
    work = torch.empty(7 * z.size, device="cuda")
    nz, ny, nx = shape
    oat.oat_tv_prox(nx, ny, nz, zt.data_ptr(), gt.data_ptr() if with_grad else None, step if with_grad else 0.0,
                    lam, iters, out.data_ptr(), work.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), want) <= 1e-5


def test_vector_kernels(env):
    torch, oat = env
    rng = np.random.default_rng(5)
    n = 100_003
    a, b, c = (rng.standard_normal(n).astype(np.float32) for _ in range(3))
    ta, tb, tc = (torch.from_numpy(v).cuda() for v in (a, b, c))
    acc = torch.zeros(4, dtype=torch.float64, device="cuda")
    r = torch.empty_like(ta)
    s = torch.cuda.current_stream().cuda_stream
    oat.oat_fista_residual(n, ta.data_ptr(), tb.data_ptr(), tc.data_ptr(), oat.OAT_F32, 0.37, r.data_ptr(),
                           acc.data_ptr(), s)
    torch.cuda.synchronize()
    a64, b64, c64 = (v.astype(np.float64) for v in (a, b, c))
    assert rel(r.cpu().numpy(), 1.37 * a64 - 0.37 * b64 - c64) <= 1e-6
    assert float(acc[0]) == pytest.approx(((a64 - c64) ** 2).sum(), rel=1e-12)
    assert float(acc[1]) == pytest.approx((c64 ** 2).sum(), rel=1e-12)
    acc.zero_()
    oat.oat_dot(n, ta.data_ptr(), tb.data_ptr(), acc.data_ptr(), s)
    y = torch.empty_like(ta)
    oat.oat_fista_momentum(n, ta.data_ptr(), tb.data_ptr(), 0.6, y.data_ptr(), s)
    torch.cuda.synchronize()
    assert float(acc[0]) == pytest.approx((a64 * b64).sum(), rel=1e-12)
    assert rel(y.cpu().numpy(), a64 + 0.6 * (a64 - b64)) <= 1e-6
    vol = rng.random((7, 9, 11)).astype(np.float32)
    acc.zero_()
    oat.oat_tv_value(11, 9, 7, torch.from_numpy(vol).cuda().data_ptr(), acc.data_ptr(), s)
    torch.cuda.synchronize()
    assert float(acc[0]) == pytest.approx(recon.tv(vol), rel=1e-6)


def test_fista_matches_reference(env):
    """Same iterations on the GPU (FP32 operators, FP64 scalars) and in the FP64 reference."""
    torch, oat = env
    from paper_1304_2017_gb300.fista import FistaTV
    geom = W.make_geometry(16, 0.3, 3, 4, 7.0, 64)
    truth = W.spheres_phantom(geom, 3, seed=12)
    u = oracle.H(geom, truth)
    plan = oat.Plan(geom)
    solver = FistaTV(plan, mu=2e-3, inner=8)
    L = solver.lipschitz(iters=40)
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    x, info = solver.solve(ut, iters=6)
    xr, res_ref = recon.fista_tv(lambda v: oracle.H(geom, v), lambda v: oracle.Ht(geom, v), u, 2e-3, L, 6,
                                 np.zeros(geom.vol_shape), inner=8)
    assert rel(x.cpu().numpy(), xr) <= 1e-4
    assert np.allclose(info["residual"], res_ref, rtol=1e-4)
    assert res_ref[-1] < res_ref[0]
    plan.close()


@pytest.mark.parametrize("name,unit", [("float32", 2.0 ** -24), ("float16", 2.0 ** -11), ("bfloat16", 2.0 ** -8)])
def test_fista_data_storage_against_reference(env, name, unit):
    """Measured data (3% Gaussian noise) stored as float32 / float16 / bfloat16, FP32 iteration
    with FP64 reductions: the final iterate against the FP64 reference run on the unrounded data.
    The difference is the storage rounding carried through (bounded here by 4 units of the
    format, plus the FP32 parity tolerance)."""
    torch, oat = env
    from paper_1304_2017_gb300.fista import FistaTV
    geom = W.make_geometry(16, 0.3, 3, 4, 7.0, 64)
    truth = W.spheres_phantom(geom, 3, seed=12)
    u = oracle.H(geom, truth)
    rng = np.random.default_rng(14)
    u = u + 0.03 * np.abs(u).max() * rng.standard_normal(u.shape)
    plan = oat.Plan(geom)
    solver = FistaTV(plan, mu=2e-3, inner=8)
    L = solver.lipschitz(iters=40)
    ut = torch.from_numpy(u.astype(np.float32)).cuda().to(getattr(torch, name))
    x, _ = solver.solve(ut, iters=6)
    xr, _ = recon.fista_tv(lambda v: oracle.H(geom, v), lambda v: oracle.Ht(geom, v), u, 2e-3, L, 6,
                           np.zeros(geom.vol_shape), inner=8)
    err = rel(x.cpu().numpy(), xr)
    print(name, "final reconstruction: rel L2 vs FP64 reference", err)
    assert err <= 4 * unit + 1e-4
    plan.close()


def test_fista_reaches_residual_target(env):
    """Noise-free, overdetermined data (64 transducers x 96 samples for 16^3 unknowns), zero
    start: the relative data residual falls to 1e-3 (the FP64 reference needs 106 iterations)."""
    torch, oat = env
    from paper_1304_2017_gb300.fista import FistaTV
    geom = W.make_geometry(16, 0.3, 8, 8, 7.0, 96)
    truth = W.spheres_phantom(geom, 3, seed=13)
    plan = oat.Plan(geom)
    u = plan.project(torch.from_numpy(truth).cuda())
    solver = FistaTV(plan, mu=1e-6, inner=5)
    x, info = solver.solve(u, iters=300, tol=1e-3)
    assert info["residual"][-1] <= 1e-3, info["residual"][-5:]
    plan.close()


def test_autograd_gradient_against_fp64_finite_differences(env):
    """d/dalpha <v, H alpha> from the autograd wrapper (backward = the adjoint kernel) against
    central differences of the FP64 oracle along random directions (32^3, 8 x 8 transducers,
    K = 128)."""
    torch, oat = env
    from paper_1304_2017_gb300 import autograd
    geom = W.config("c3_grad")
    plan = oat.Plan(geom)
    alpha = W.spheres_phantom(geom, 4, seed=14)
    v = W.random_data(geom, seed=15)
    a = torch.from_numpy(alpha).cuda().requires_grad_(True)
    loss = (autograd.project(a, plan).double() * torch.from_numpy(v).cuda().double()).sum()
    loss.backward()
    grad = a.grad.detach().cpu().numpy().astype(np.float64)
    assert rel(grad, oracle.Ht(geom, v)) <= 1e-5
    rng = np.random.default_rng(16)
    eps = 1e-3
    for _ in range(3):
        e = rng.standard_normal(geom.vol_shape)
        fp = (v * oracle.H(geom, alpha + eps * e)).sum()
        fm = (v * oracle.H(geom, alpha - eps * e)).sum()
        fd = (fp - fm) / (2 * eps)
        # random directions make <grad, e> a cancelling sum: normalise as the adjoint identity
        assert abs((grad * e).sum() - fd) <= 1e-5 * np.linalg.norm(grad) * np.linalg.norm(e)
    # backward of the backprojection is the projector
    y = torch.from_numpy(v).cuda().requires_grad_(True)
    w = torch.from_numpy(alpha).cuda().double()
    (autograd.backproject(y, plan).double() * w).sum().backward()
    gy = y.grad.detach().cpu().numpy().astype(np.float64)
    assert rel(gy, oracle.H(geom, alpha)) <= 1e-5
    plan.close()
