"""Parity of the projector / backprojector with exact strip-area lattice weights
(OAT_LATTICE_EXACT_AREA: point weight Delta_s 2 pi rho sin(theta_i) / N_j instead of Delta_s^2)
against the FP64 oracle with the same weights.

Tolerance 1e-5 relative L2 and for the adjoint identity, as with uniform weights: the kernels
multiply each point's interpolated value (or its g') by its ring's weight factor, rounded once to
float32 from the FP64 table."""
import dataclasses

import numpy as np
import pytest

import oracle
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
    return torch, oat


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def area(g):
    return dataclasses.replace(g, lattice_weights=1)


def run(env, geom, alpha, y, dtype=0, apply_d=True):
    torch, oat = env
    plan = oat.Plan(geom, data_dtype=dtype, apply_d=apply_d)
    try:
        u = plan.project(torch.from_numpy(np.ascontiguousarray(alpha, np.float32)).cuda())
        yt = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda().to(plan.torch_data_dtype)
        a = plan.backproject(yt)
        torch.cuda.synchronize()
        return u.float().cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64), yt.float().cpu().numpy()
    finally:
        plan.close()


CASES = {
    "small_ragged": lambda: W.config("small"),
    "tmin0": lambda: W.make_geometry(18, 0.3, 2, 3, 6.0, 100, t_min_us=0.0),
    "partial_window": lambda: W.make_geometry(16, 0.3, 3, 3, 8.0, 40),
    "offset_grid": lambda: W.make_geometry((14, 19, 11), 0.35, 3, 5, 9.0, 110, origin_mm=(-3.1, -2.2, -1.4)),
    "on_axis": lambda: W.make_geometry(12, 0.3, 2, 2, 7.0, 80,
                                       positions_mm=[[0, 0, 7.0], [0, 0, -7.5], [7.2, 0, 0], [0, 6.9, 0.3]]),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("apply_d", [True, False])
def test_area_matches_reference(env, case, apply_d):
    geom = area(CASES[case]())
    alpha = W.spheres_phantom(geom, 4, seed=3) + 0.05 * W.random_volume(geom, seed=4)
    y = W.random_data(geom, seed=5)
    u, a, yq = run(env, geom, alpha, y, apply_d=apply_d)
    u_ref = oracle.H(geom, alpha, apply_d=apply_d)
    a_ref = oracle.Ht(geom, yq, apply_d=apply_d)
    lhs = float((u * yq).sum()); rhs = float((alpha.astype(np.float64) * a).sum())
    errs = (rel(u, u_ref), rel(a, a_ref), abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(yq)))
    # the weights matter here: the uniform-weight reference is far away
    far = rel(oracle.H(dataclasses.replace(geom, lattice_weights=0), alpha, apply_d=apply_d), u_ref)
    print(case, apply_d, errs, "uniform vs area", far)
    assert far > 1e-3
    assert max(errs) <= TOL, errs


def test_area_dense_tiny(env):
    geom = area(W.config("tiny"))
    M = oracle.dense_G(geom)
    alpha = W.random_volume(geom, seed=1)
    y = W.random_data(geom, seed=2)
    u, a, yq = run(env, geom, alpha, y, apply_d=False)
    assert rel(u.ravel(), M @ alpha.astype(np.float64).ravel()) <= TOL
    assert rel(a.ravel(), M.T @ yq.astype(np.float64).ravel()) <= TOL


@pytest.mark.parametrize("dtype,store", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_area_half_storage(env, dtype, store):
    geom = area(W.make_geometry(24, 0.25, 3, 4, 8.0, 96))
    alpha = W.spheres_phantom(geom, 4, seed=8)
    y = W.random_data(geom, seed=9)
    u, a, yq = run(env, geom, alpha, y, dtype=dtype)
    assert rel(u, oracle.H(geom, alpha)) <= store + TOL
    assert rel(a, oracle.Ht(geom, yq)) <= TOL


def test_area_full_size(env):
    """256^3, 23,040 transducers, K = 1536 with exact strip areas: the rows of four sampled
    transducers, H^T of data on them alone, and the adjoint identity with dense data."""
    torch, oat = env
    geom = area(W.config("c2"))
    qs = [0, 64 * 180 + 45, 100 * 180 + 137, 23039]
    sub = geom.subset(qs)
    alpha = W.phantom("c2", geom)
    plan = oat.Plan(geom)
    try:
        u = plan.project(torch.from_numpy(alpha).cuda())
        errs = {"H": rel(u[qs].cpu().numpy(), oracle.H(sub, alpha))}
        y = torch.zeros(geom.data_shape, device="cuda")
        y_s = W.random_data(sub, seed=31)
        y[qs] = torch.from_numpy(y_s).cuda()
        errs["Ht"] = rel(plan.backproject(y).cpu().numpy(), oracle.Ht(sub, y_s))
        yd = torch.from_numpy(W.random_data(geom, seed=32)).cuda()
        ad = plan.backproject(yd)
        lhs = float((u.double() * yd.double()).sum())
        rhs = float((torch.from_numpy(alpha).cuda().double() * ad.double()).sum())
        errs["adjoint"] = abs(lhs - rhs) / (float(u.double().norm()) * float(yd.double().norm()))
        torch.cuda.synchronize()
    finally:
        plan.close()
    print("area full size", errs)
    assert max(errs.values()) <= TOL, errs
