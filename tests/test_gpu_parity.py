"""Parity of the sm_103a projector / backprojector (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 error <= 1e-5 for FP32 data, and the adjoint identity
|<Hx, y> - <x, H^T y>| / (||Hx|| ||y||) <= 1e-5 with FP64 reductions.  For FP16 / BF16 data
storage the projector's tolerance adds the storage rounding (2^-11 resp. 2^-8 relative); the
backprojector reads the stored values exactly, so its tolerance stays 1e-5."""
import numpy as np
import pytest

import oracle
from paper_1304_2017_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def oat(torch_cuda):
    from paper_1304_2017_gb300 import oat as mod
    return mod


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(oat, torch, geom, alpha, y, dtype=0, apply_d=True):
    plan = oat.Plan(geom, data_dtype=dtype, apply_d=apply_d)
    u = plan.project(torch.from_numpy(np.ascontiguousarray(alpha, np.float32)).cuda())
    yt = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda().to(plan.torch_data_dtype)
    a = plan.backproject(yt)
    torch.cuda.synchronize()
    out = u.float().cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64), yt.float().cpu().numpy()
    plan.close()
    return out


def adjoint_err(u, y, alpha, a):
    lhs = float((u * y).sum())
    rhs = float((alpha.astype(np.float64) * a).sum())
    return abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(y))


CASES = {
    "tiny": lambda: W.config("tiny"),
    "small_ragged": lambda: W.config("small"),
    "tmin0": lambda: W.make_geometry(18, 0.3, 2, 3, 6.0, 100, t_min_us=0.0),
    "flat_z": lambda: W.make_geometry((23, 17, 1), 0.3, 3, 4, 9.0, 90),
    "single_xdcr_k3": lambda: W.make_geometry(10, 0.4, 1, 1, 6.0, 3, t_min_us=6.0 / 1.5 - 0.05),
    "on_axis": lambda: W.make_geometry(12, 0.3, 2, 2, 7.0, 80,
                                       positions_mm=[[0, 0, 7.0], [0, 0, -7.5], [7.2, 0, 0], [0, 6.9, 0.3]]),
    "partial_window": lambda: W.make_geometry(16, 0.3, 3, 3, 8.0, 40),
    "offset_grid": lambda: W.make_geometry((14, 19, 11), 0.35, 3, 5, 9.0, 110, origin_mm=(-3.1, -2.2, -1.4)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("apply_d", [True, False])
def test_parity_small_cases(oat, torch_cuda, case, apply_d):
    geom = CASES[case]()
    alpha = W.spheres_phantom(geom, 4, seed=3) + 0.05 * W.random_volume(geom, seed=4)
    y = W.random_data(geom, seed=5)
    u, a, yq = run(oat, torch_cuda, geom, alpha, y, apply_d=apply_d)
    u_ref = oracle.H(geom, alpha, apply_d=apply_d)
    a_ref = oracle.Ht(geom, yq, apply_d=apply_d)
    assert np.abs(u_ref).max() > 0
    assert rel(u, u_ref) <= TOL, rel(u, u_ref)
    assert rel(a, a_ref) <= TOL, rel(a, a_ref)
    assert adjoint_err(u, yq, alpha, a) <= TOL


def test_dense_matrix_tiny(oat, torch_cuda):
    """GPU H and H^T against the brute-force dense matrix (P-dense)."""
    geom = W.config("tiny")
    M = oracle.dense_G(geom)
    alpha = W.random_volume(geom, seed=1)
    y = W.random_data(geom, seed=2)
    u, a, yq = run(oat, torch_cuda, geom, alpha, y, apply_d=False)
    assert rel(u.ravel(), M @ alpha.astype(np.float64).ravel()) <= TOL
    assert rel(a.ravel(), M.T @ yq.astype(np.float64).ravel()) <= TOL


def test_parity_c1_full(oat, torch_cuda):
    """64^3 / 256 transducers / K = 256: every output against the oracle, adjoint identity."""
    geom = W.config("c1")
    alpha = W.phantom("c1", geom)
    y = W.random_data(geom, seed=7)
    u, a, yq = run(oat, torch_cuda, geom, alpha, y)
    u_ref = oracle.H(geom, alpha)
    assert rel(u, u_ref) <= TOL, rel(u, u_ref)
    a_ref = oracle.Ht(geom, yq)
    assert rel(a, a_ref) <= TOL, rel(a, a_ref)
    assert adjoint_err(u, yq, alpha, a) <= TOL


@pytest.mark.parametrize("dtype,name", [(1, "f16"), (2, "bf16")])
def test_half_storage(oat, torch_cuda, dtype, name):
    geom = W.make_geometry(24, 0.25, 3, 4, 8.0, 96)
    alpha = W.spheres_phantom(geom, 4, seed=8)
    y = W.random_data(geom, seed=9)
    u, a, yq = run(oat, torch_cuda, geom, alpha, y, dtype=dtype)
    u_ref = oracle.H(geom, alpha)
    store = {1: 2.0 ** -11, 2: 2.0 ** -8}[dtype]
    assert rel(u, u_ref) <= store + TOL, (name, rel(u, u_ref))
    a_ref = oracle.Ht(geom, yq)
    assert rel(a, a_ref) <= TOL, (name, rel(a, a_ref))


def test_point_count_matches_oracle(oat, torch_cuda):
    geom = W.config("c1")
    plan = oat.Plan(geom)
    st = plan.stats(count_grid_points=True)
    nb, ng = oracle.count_points(geom)
    assert st["points_ball"] == nb
    assert abs(st["points_grid"] - ng) <= 1e-6 * ng + 2
    plan.close()


def test_misaligned_and_wrong_args(oat, torch_cuda):
    torch = torch_cuda
    geom = W.make_geometry(10, 0.4, 1, 2, 6.0, 32)
    plan = oat.Plan(geom)
    buf = torch.zeros(geom.n_voxels + 4, device="cuda")
    dat = torch.zeros(geom.n_transducers * geom.n_samples + 4, device="cuda")
    with pytest.raises(oat.OatError) as e:
        oat.oat_project(plan.handle, buf.data_ptr() + 4, dat.data_ptr(), 0)
    assert e.value.code == oat.OAT_ERR_INVALID_ARG
    with pytest.raises(oat.OatError):
        oat.oat_backproject(plan.handle, dat.data_ptr() + 8, buf.data_ptr(), 0)
    with pytest.raises(ValueError):
        plan.project(torch.zeros(3, 3, 3, device="cuda"))
    plan.close()


def test_repeat_calls_deterministic_and_stream(oat, torch_cuda):
    """Repeated calls on a side stream give identical results (no atomics in either direction)."""
    torch = torch_cuda
    geom = W.config("small")
    alpha = torch.from_numpy(W.phantom("small", geom)).cuda()
    y = torch.from_numpy(W.random_data(geom)).cuda()
    plan = oat.Plan(geom)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u1 = plan.project(alpha); a1 = plan.backproject(y)
        u2 = plan.project(alpha); a2 = plan.backproject(y)
    s.synchronize()
    assert torch.equal(u1, u2) and torch.equal(a1, a2)
    plan.close()


def test_plan_reuse_after_other_inputs(oat, torch_cuda):
    """A plan reused with new inputs (including shells that hold no lattice point, whose
    sums no work item writes) gives the oracle's result for the new inputs."""
    torch = torch_cuda
    geom = CASES["partial_window"]()
    plan = oat.Plan(geom)
    a1 = W.random_volume(geom, seed=21) * 10
    a2 = W.spheres_phantom(geom, 3, seed=22)
    y1 = W.random_data(geom, seed=23) * 5
    y2 = W.random_data(geom, seed=24)
    plan.project(torch.from_numpy(a1).cuda()); plan.backproject(torch.from_numpy(y1).cuda())
    u = plan.project(torch.from_numpy(a2).cuda()).cpu().numpy()
    a = plan.backproject(torch.from_numpy(y2).cuda()).cpu().numpy()
    assert rel(u, oracle.H(geom, a2)) <= TOL
    assert rel(a, oracle.Ht(geom, y2)) <= TOL
    plan.close()
