"""Parity of the sm_103a spherical-voxel model (oat_sph_project / oat_sph_backproject, through the
C ABI) with the FP64 reference oracle/sph.py (Eqs. dis_sph, p0f, sphbwd).

Tolerance 1e-5 relative L2 for u = H_sph alpha (complex), for alpha' = H_sph^T u, and for the
adjoint identity Re <H alpha, u> = <alpha, H^T u>: phases are formed from float-pair distances
(about 1e-10 cycle), consecutive frequencies by short complex rotations (a few 1e-7), and sums
are compensated."""
import math

import numpy as np
import pytest

from oracle import sph as S
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = {
    # (geometry, L, f0, df): the paper's band (0, 5] MHz sampled as f_l = (l + 1) 5 / L
    "ragged_L37": (lambda: W.make_geometry((9, 7, 8), 0.3, 2, 3, 6.0, 16), 37, 5.0 / 37, 5.0 / 37),
    "two_runs_L300": (lambda: W.make_geometry((11, 6, 5), 0.25, 3, 4, 5.0, 16), 300, 5.0 / 300, 5.0 / 300),
    "far_65mm_L511": (lambda: W.make_geometry(12, 0.2, 2, 3, 65.0, 16), 511, 5.0 / 511, 5.0 / 511),
    "single_freq": (lambda: W.make_geometry((6, 5, 7), 0.3, 2, 2, 5.0, 16), 1, 2.3, 0.0),
    "offset_band": (lambda: W.make_geometry((8, 8, 3), 0.2, 2, 3, 7.0, 16, gruneisen=1.7), 70, 0.8, 0.031),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sph_matches_reference(env, case):
    torch, oat = env
    make, L, f0, df = CASES[case]
    geom = make()
    rng = np.random.default_rng(7)
    alpha = (W.spheres_phantom(geom, 3, seed=2) + 0.1 * rng.standard_normal(geom.vol_shape)).astype(np.float32)
    u_in = (rng.standard_normal((geom.n_transducers, L)) + 1j * rng.standard_normal((geom.n_transducers, L)))
    u_in = u_in.astype(np.complex64)
    op = oat.SphOp(geom, L, f0, df)
    try:
        u = op.project(torch.from_numpy(alpha).cuda()).cpu().numpy()
        a = op.backproject(torch.from_numpy(u_in).cuda()).cpu().numpy()
        torch.cuda.synchronize()
    finally:
        op.close()
    freqs = f0 + df * np.arange(L)
    u_ref = S.H_sph(geom, alpha, freqs)
    a_ref = S.H_sph_t(geom, u_in, freqs)
    lhs = float(np.real(np.vdot(u.astype(np.complex128), u_in.astype(np.complex128))))
    rhs = float((alpha.astype(np.float64) * a.astype(np.float64)).sum())
    errs = (rel(u, u_ref), rel(a, a_ref), abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(u_in)))
    print(case, errs)
    assert max(errs) <= TOL, errs


def test_sph_with_eir_and_bad_args(env):
    torch, oat = env
    geom = W.make_geometry((7, 6, 5), 0.3, 2, 3, 6.0, 16)
    L, f0, df = 40, 0.1, 0.12
    rng = np.random.default_rng(3)
    eir = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    alpha = rng.standard_normal(geom.vol_shape).astype(np.float32)
    u_in = (rng.standard_normal((geom.n_transducers, L)) + 1j * rng.standard_normal((geom.n_transducers, L)))
    u_in = u_in.astype(np.complex64)
    op = oat.SphOp(geom, L, f0, df, eir=eir)
    try:
        u = op.project(torch.from_numpy(alpha).cuda()).cpu().numpy()
        a = op.backproject(torch.from_numpy(u_in).cuda()).cpu().numpy()
    finally:
        op.close()
    freqs = f0 + df * np.arange(L)
    assert rel(u, S.H_sph(geom, alpha, freqs, eir=eir)) <= TOL
    assert rel(a, S.H_sph_t(geom, u_in, freqs, eir=eir)) <= TOL
    # a transducer on a node, a non-positive frequency, a zero step with several frequencies
    bad = W.make_geometry(6, 0.3, 1, 1, 5.0, 16, positions_mm=[[0.15, 0.15, 0.15]])
    for g_, args in ((bad, (4, 0.5, 0.1)), (geom, (4, 0.0, 0.1)), (geom, (4, 0.5, 0.0))):
        with pytest.raises(oat.OatError) as e:
            oat.SphOp(g_, *args)
        assert e.value.code == oat.OAT_ERR_INVALID_ARG


def test_sph_maximum_frequency_count(env):
    """L = 12,800, the largest the adjoint's shared-memory staging takes (one transducer row of
    packed values per tile, 200 KB): both directions against the reference on a small grid."""
    torch, oat = env
    geom = W.make_geometry((4, 3, 5), 0.3, 1, 2, 5.0, 16)
    L, f0, df = 12800, 0.01, 5.0 / 12800
    rng = np.random.default_rng(21)
    alpha = rng.standard_normal(geom.vol_shape).astype(np.float32)
    u_in = (rng.standard_normal((geom.n_transducers, L)) + 1j * rng.standard_normal((geom.n_transducers, L)))
    u_in = u_in.astype(np.complex64)
    op = oat.SphOp(geom, L, f0, df)
    try:
        u = op.project(torch.from_numpy(alpha).cuda()).cpu().numpy()
        a = op.backproject(torch.from_numpy(u_in).cuda()).cpu().numpy()
    finally:
        op.close()
    freqs = f0 + df * np.arange(L)
    errs = (rel(u, S.H_sph(geom, alpha, freqs)), rel(a, S.H_sph_t(geom, u_in, freqs)))
    print("sph L = 12800", errs)
    assert max(errs) <= TOL, errs
    with pytest.raises(oat.OatError):
        oat.SphOp(geom, 12801, f0, df)


def test_sph_full_size_sampled(env):
    """The paper's simulation scale: 210 x 210 x 440 nodes at 0.14 mm, 64 rings x 90 views on 65 mm,
    511 frequencies in (0, 5] MHz.  Sampled outputs against the reference: u at 3 transducers x 4
    frequencies (each a sum over all 19.4 M voxels), alpha' at 12 nodes (each a sum over all
    5,760 x 511 data)."""
    torch, oat = env
    geom = W.sph_config()
    L, f0, df = 511, 5.0 / 511, 5.0 / 511
    alpha = W.phantom_sph(geom)
    rng = np.random.default_rng(11)
    u_in = (rng.standard_normal((geom.n_transducers, L)) + 1j * rng.standard_normal((geom.n_transducers, L)))
    u_in = u_in.astype(np.complex64)
    op = oat.SphOp(geom, L, f0, df)
    try:
        u = op.project(torch.from_numpy(alpha).cuda()).cpu().numpy()
        a = op.backproject(torch.from_numpy(u_in).cuda()).cpu().numpy()
    finally:
        op.close()
    freqs = f0 + df * np.arange(L)
    qs, ls = [0, 2000, 5759], [0, 100, 333, 510]
    u_ref = S.H_sph(geom, alpha, freqs[ls], qs=qs)
    nodes = np.stack([rng.integers(0, n, 12) for n in (geom.nx, geom.ny, geom.nz)], axis=1)
    nodes[0] = 0
    nodes[1] = (geom.nx - 1, geom.ny - 1, geom.nz - 1)
    a_ref = S.H_sph_t(geom, u_in, freqs, nodes=nodes)
    errs = (rel(u[np.ix_(qs, ls)], u_ref), rel(a[nodes[:, 2], nodes[:, 1], nodes[:, 0]], a_ref))
    print("sph full size", errs)
    assert max(errs) <= TOL, errs
