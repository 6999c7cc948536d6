"""Parity of the projector / backprojector with a transducer response (oat_plan_set_eir, Sec. II.B,
Eq. EIR) against the FP64 references: H = H^e D G is oracle.H followed by oracle/eir.Heir, and
H^T = G^T D^T H^e^T is oracle/eir.Heir_t followed by oracle.Ht.

Tolerance 1e-5 relative L2 and for the adjoint identity, as without a response: both kernels
keep D G alpha and the convolution in double precision and round once."""
import numpy as np
import pytest

import oracle
from oracle import eir as E
from eir_conv import conv_rows, corr_rows
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


def adjoint_err(u, y, alpha, a):
    lhs = float((np.asarray(u, np.float64) * y).sum())
    rhs = float((alpha.astype(np.float64) * a).sum())
    return abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(y))


GEOMS = {
    "small_ragged": lambda: W.config("small"),
    "tmin0": lambda: W.make_geometry(18, 0.3, 2, 3, 6.0, 100, t_min_us=0.0),
    "partial_window": lambda: W.make_geometry(16, 0.3, 3, 3, 8.0, 40),
}
RESPONSES = {
    "gaussian": lambda: W.eir_taps(kind="gaussian"),
    "bandpass": lambda: W.eir_taps(kind="bandpass"),
    # taps reaching past both ends of a short record
    "wide_offset": lambda: (np.random.default_rng(4).standard_normal(61) / 61.0, -45),
}


def run(env, geom, h, m0, alpha, y, dtype=0, apply_d=True):
    torch, oat = env
    plan = oat.Plan(geom, data_dtype=dtype, apply_d=apply_d)
    try:
        plan.set_eir(h, m0)
        u = plan.project(torch.from_numpy(np.ascontiguousarray(alpha, np.float32)).cuda())
        yt = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda().to(plan.torch_data_dtype)
        a = plan.backproject(yt)
        torch.cuda.synchronize()
        return u.float().cpu().numpy().astype(np.float64), a.cpu().numpy().astype(np.float64), yt.float().cpu().numpy()
    finally:
        plan.close()


@pytest.mark.parametrize("geom_name", sorted(GEOMS))
@pytest.mark.parametrize("resp", sorted(RESPONSES))
def test_eir_matches_reference(env, geom_name, resp):
    geom = GEOMS[geom_name]()
    h, m0 = RESPONSES[resp]()
    alpha = W.spheres_phantom(geom, 4, seed=3) + 0.05 * W.random_volume(geom, seed=4)
    y = W.random_data(geom, seed=5)
    u, a, yq = run(env, geom, h, m0, alpha, y)
    u_ref = E.Heir(oracle.H(geom, alpha), h, m0)
    a_ref = oracle.Ht(geom, E.Heir_t(yq, h, m0))
    assert np.abs(u_ref).max() > 0 and np.abs(a_ref).max() > 0
    errs = (rel(u, u_ref), rel(a, a_ref), adjoint_err(u, yq, alpha, a))
    print(geom_name, resp, errs)
    assert errs[0] <= TOL and errs[1] <= TOL and errs[2] <= TOL, errs


def test_eir_without_d(env):
    geom = W.config("small")
    h, m0 = W.eir_taps(kind="bandpass")
    alpha = W.spheres_phantom(geom, 4, seed=6)
    y = W.random_data(geom, seed=7)
    u, a, yq = run(env, geom, h, m0, alpha, y, apply_d=False)
    assert rel(u, E.Heir(oracle.H(geom, alpha, apply_d=False), h, m0)) <= TOL
    assert rel(a, oracle.Ht(geom, E.Heir_t(yq, h, m0), apply_d=False)) <= TOL


@pytest.mark.parametrize("dtype,store", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_eir_half_storage(env, dtype, store):
    """FP16 / BF16 data: H^e D G alpha rounded once to the storage type; H^T reads the stored
    values exactly."""
    geom = W.make_geometry(24, 0.25, 3, 4, 8.0, 96)
    h, m0 = W.eir_taps(kind="gaussian")
    alpha = W.spheres_phantom(geom, 4, seed=8)
    y = W.random_data(geom, seed=9)
    u, a, yq = run(env, geom, h, m0, alpha, y, dtype=dtype)
    assert rel(u, E.Heir(oracle.H(geom, alpha), h, m0)) <= store + TOL
    assert rel(a, oracle.Ht(geom, E.Heir_t(yq, h, m0))) <= TOL


def test_identity_response_and_removal(env):
    """h_{-1} = 1 is the identity (Eq. EIR's one-sample offset cancels): the results equal those
    without a response bit for bit; removing the response (no taps) restores the plain model."""
    torch, oat = env
    geom = W.config("small")
    alpha = torch.from_numpy(W.spheres_phantom(geom, 4, seed=10)).cuda()
    y = torch.from_numpy(W.random_data(geom, seed=11)).cuda()
    plan = oat.Plan(geom)
    try:
        u0, a0 = plan.project(alpha).clone(), plan.backproject(y).clone()
        plan.set_eir([1.0], -1)
        u1, a1 = plan.project(alpha).clone(), plan.backproject(y).clone()
        plan.set_eir([0.5], 0)
        u2 = plan.project(alpha).clone()
        plan.set_eir([])
        u3, a3 = plan.project(alpha).clone(), plan.backproject(y).clone()
        torch.cuda.synchronize()
    finally:
        plan.close()
    assert torch.equal(u0, u1) and torch.equal(a0, a1)
    assert torch.equal(u0, u3) and torch.equal(a0, a3)
    # h_0 = 0.5: a one-sample delay, halved (exact in binary)
    assert torch.equal(u2[:, 1:], 0.5 * u0[:, :-1]) and bool((u2[:, 0] == 0).all())


def test_eir_bad_args(env):
    torch, oat = env
    geom = W.make_geometry(8, 0.4, 2, 2, 6.0, 32)
    plan = oat.Plan(geom)
    try:
        with pytest.raises(oat.OatError) as e:
            plan.set_eir([1.0, float("nan")], 0)
        assert e.value.code == oat.OAT_ERR_INVALID_ARG
        with pytest.raises(oat.OatError):
            plan.set_eir([1.0], (1 << 30) + 1)
        with pytest.raises(oat.OatError):
            plan.set_eir(np.ones(40000), 0)
    finally:
        plan.close()


def test_eir_long_record_near_the_shared_memory_bound(env):
    """K = 20,000 samples at 20 MHz with 7,000 taps: (K + taps) doubles = 216 KB of a block's shared memory
    (the bound is the device's opt-in maximum, 227 KB on GB300)."""
    torch, oat = env
    geom = W.make_geometry(6, 0.5, 1, 2, 6.0, 20000, t_min_us=0.0)
    rng = np.random.default_rng(8)
    h = rng.standard_normal(7000) / 7000.0
    m0 = -3500
    alpha = W.spheres_phantom(geom, 2, seed=3, r_range=(0.4, 0.9))
    y = W.random_data(geom, seed=4)
    u, a, yq = run(env, geom, h, m0, alpha, y)
    errs = (rel(u, conv_rows(oracle.H(geom, alpha), h, m0)),
            rel(a, oracle.Ht(geom, corr_rows(yq.astype(np.float64), h, m0))))
    print("eir K = 20000", errs)
    assert max(errs) <= TOL, errs


def test_eir_full_size(env):
    """256^3, 23,040 transducers, K = 1536, the simulation studies' Gaussian response: the rows
    of four sampled transducers, H^T of data on them alone, and the adjoint identity with
    dense data."""
    torch, oat = env
    geom = W.config("c2")
    qs = [0, 64 * 180 + 45, 100 * 180 + 137, 23039]
    sub = geom.subset(qs)
    h, m0 = W.eir_taps(kind="gaussian")
    alpha = W.phantom("c2", geom)
    plan = oat.Plan(geom)
    try:
        plan.set_eir(h, m0)
        u = plan.project(torch.from_numpy(alpha).cuda())
        errs = {"H": rel(u[qs].cpu().numpy(), E.Heir(oracle.H(sub, alpha), h, m0))}
        y = torch.zeros(geom.data_shape, device="cuda")
        y_s = W.random_data(sub, seed=31)
        y[qs] = torch.from_numpy(y_s).cuda()
        errs["Ht"] = rel(plan.backproject(y).cpu().numpy(), oracle.Ht(sub, E.Heir_t(y_s, h, m0)))
        yd = torch.from_numpy(W.random_data(geom, seed=32)).cuda()
        ad = plan.backproject(yd)
        lhs = float((u.double() * yd.double()).sum())
        rhs = float((torch.from_numpy(alpha).cuda().double() * ad.double()).sum())
        errs["adjoint"] = abs(lhs - rhs) / (float(u.double().norm()) * float(yd.double().norm()))
        torch.cuda.synchronize()
    finally:
        plan.close()
    print("eir full size", errs)
    assert max(errs.values()) <= TOL, errs
