"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute-force dense matrices built from the definition of psi_n, scipy's trilinear
interpolation, closed forms of the continuous model, exact identities of the lattice,
and the symmetry of the scanner.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_1304_2017_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------------------------ dense

def test_dense_brute_force_equals_fast_G_and_scatter_Gt():
    """P-dense: H assembled column by column from psi_n's definition (every node, no
    8-neighbour shortcut) equals the oracle's trilinear G and its scatter transpose."""
    g = W.config("tiny")
    M = oracle.dense_G(g)
    assert M.shape == (g.n_transducers * g.n_samples, g.n_voxels)
    assert np.count_nonzero(M) > 100
    x = W.random_volume(g, seed=3).astype(np.float64)
    y = W.random_data(g, seed=4).astype(np.float64)
    gx = oracle.G(g, x)
    assert _rel(gx.ravel(), M @ x.ravel()) < 1e-12
    gty = oracle.Gt(g, y)
    assert _rel(gty.ravel(), M.T @ y.ravel()) < 1e-12
    # H = D G: with the dense D built from unit vectors
    K = g.n_samples
    Dm = np.zeros((K, K))
    sub = g.subset([0])
    for j in range(K):
        e = np.zeros((1, K)); e[0, j] = 1.0
        Dm[:, j] = oracle.D(sub, e)[0]
    Hd = np.kron(np.eye(g.n_transducers), Dm) @ M
    assert _rel(oracle.H(g, x).ravel(), Hd @ x.ravel()) < 1e-12
    assert _rel(oracle.Ht(g, y).ravel(), Hd.T @ y.ravel()) < 1e-12


def test_dense_non_cubic_offset_grid():
    """Same brute force on a non-cubic grid whose origin is not centred (transposed axes or a
    wrong origin would break it)."""
    g = W.make_geometry((5, 4, 7), 0.45, 2, 3, 7.0, 30, fs_mhz=12.0, origin_mm=(-1.3, -0.6, -1.1))
    M = oracle.dense_G(g)
    x = W.random_volume(g, seed=5).astype(np.float64)
    assert np.count_nonzero(M) > 50
    assert _rel(oracle.G(g, x).ravel(), M @ x.ravel()) < 1e-12


# ------------------------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("tmin", [None, 0.0])
def test_adjoint_identity(tmin):
    """P-adjoint: <H x, y> = <x, H^T y> to rounding (FP64)."""
    g = W.make_geometry(24, 0.25, 4, 4, 8.0, 96, t_min_us=tmin)
    x = W.spheres_phantom(g, 4, seed=1).astype(np.float64)
    y = W.random_data(g, seed=2).astype(np.float64)
    hx = oracle.H(g, x)
    hty = oracle.Ht(g, y)
    lhs, rhs = float((hx * y).sum()), float((x * hty).sum())
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(hx) * np.linalg.norm(y)


@pytest.mark.parametrize("tmin", [0.0, 0.05, 3.0])
def test_D_transpose(tmin):
    """P-D: <D g, p> = <g, D^T p>, including t_min = 0 (tau_0 = 0, tau_1 = 1)."""
    g = W.make_geometry(4, 0.5, 2, 2, 5.0, 37, t_min_us=tmin)
    rng = np.random.default_rng(0)
    a = rng.standard_normal(g.data_shape)
    b = rng.standard_normal(g.data_shape)
    lhs = (oracle.D(g, a) * b).sum()
    rhs = (a * oracle.Dt(g, b)).sum()
    assert abs(lhs - rhs) <= 1e-14 * np.abs(oracle.D(g, a)).sum() * np.abs(b).max() * 10


def test_D_is_derivative_of_g_over_t():
    """D approximates (Gamma/c^2)/(4 pi) d/dt (g/t) (Eq. g2p) and is exact for g = t^3:
    d/dt(t^2) = 2t, so p_k = Gamma t_k / (2 pi c^2) in the interior rows."""
    gam, c = 2000.0, 1.54
    g = W.make_geometry(4, 0.5, 1, 1, 5.0, 50, fs_mhz=20.0, c=c, t_min_us=1.3, gruneisen=gam)
    t = g.t_min_us + np.arange(g.n_samples) / g.fs_mhz
    p = oracle.D(g, (t ** 3)[None, :])[0]
    want = gam * t / (2 * math.pi * c * c)
    assert np.allclose(p[1:-1], want[1:-1], rtol=1e-11, atol=0)
    assert p[0] == 0.0 and p[-1] == 0.0


# ------------------------------------------------------------------------------------ lattice

def test_lattice_geometry():
    """Points lie on the shell |P - r_q| = c t_k inside the support sphere; consecutive points
    of a ring are one spacing apart in arc length (floor count N_j), rings are one spacing
    apart along the meridian (Appendix)."""
    g = W.config("c1")
    q, k = 37, 131
    P, ij, nr = oracle.shell_points(g, q, k)
    rq = g.positions_mm[q]
    rho = g.c_mm_per_us * (g.t_min_us + k / g.fs_mhz)
    assert len(P) > 1000
    assert np.allclose(np.linalg.norm(P - rq, axis=1), rho, rtol=0, atol=1e-11)
    assert np.all(np.linalg.norm(P, axis=1) <= g.support_radius_mm + 1e-9)
    ds = g.spacing_mm
    ez = -rq / np.linalg.norm(rq)
    cos_th = ((P - rq) @ ez) / rho
    th = np.arccos(np.clip(cos_th, -1, 1))
    assert np.allclose(th, ij[:, 0] * ds / rho, atol=1e-9)        # theta_i = i * ds / rho
    for i in np.unique(ij[:, 0]):
        sel = ij[:, 0] == i
        a = rho * math.sin(i * ds / rho)                           # ring radius
        nj = sel.sum()
        assert nj * ds <= 2 * math.pi * a + 1e-9 < (nj + 1) * ds   # N_j = floor(2 pi a / ds)
        pts = P[sel]
        chords = np.linalg.norm(np.diff(pts, axis=0), axis=1)
        assert np.allclose(chords, 2 * a * math.sin(ds / (2 * a)), rtol=1e-9)
    # number of rings N_i = floor(theta_max / dtheta): N_i dtheta <= theta_max < (N_i + 1) dtheta
    rs = np.linalg.norm(rq)
    thmax = math.acos((rs * rs + rho * rho - g.support_radius_mm ** 2) / (2 * rho * rs))
    assert nr * ds / rho <= thmax + 1e-12 and (nr + 1) * ds / rho > thmax - 1e-12
    # count vs cap area: the rings form a Riemann sum of 2 pi rho^2 sin(theta) dtheta / ds^2,
    # floor() drops less than one point per ring, so (theta <= pi/2 here)
    #   area(theta_{N_i - 1}) / ds^2 - N_i <= count <= area(theta_{N_i}) / ds^2
    dth = ds / rho
    assert nr * dth < math.pi / 2
    area = lambda th_: 2 * math.pi * rho * rho * (1 - math.cos(th_)) / ds ** 2  # noqa: E731
    assert area((nr - 1) * dth) - nr <= len(P) <= area(nr * dth)


def test_interpolation_matches_scipy():
    """The oracle's trilinear interpolant (zero outside the nodes) equals scipy's
    map_coordinates(order=1, mode='grid-constant') at the lattice points of a shell."""
    g = W.config("c1")
    a = W.phantom("c1", g).astype(np.float64)
    a += W.random_volume(g, seed=9).astype(np.float64) * 0.1
    for q, k in [(0, 100), (77, 128), (255, 170), (130, 60)]:
        P, _, _ = oracle.shell_points(g, q, k)
        idx = (P - np.asarray(g.origin_mm)) / g.spacing_mm          # (x, y, z) index coords
        f = ndimage.map_coordinates(a, idx[:, ::-1].T, order=1, mode="grid-constant", cval=0.0,
                                    prefilter=False)
        want = g.spacing_mm ** 2 * f.sum()
        got = oracle.G_rows(g, a, [(q, k)])[0]
        assert abs(got - want) <= 1e-10 * max(abs(want), 1.0), (q, k, got, want)


def test_constant_and_affine_volumes_are_exact():
    """P-count: with the support sphere inside the node cuboid, alpha = 1 gives
    g_k = ds^2 * (number of points) exactly; an affine alpha gives ds^2 * sum of the affine
    function at the points (trilinear interpolation reproduces affine functions)."""
    base = W.make_geometry(40, 0.25, 3, 4, 9.0, 200)
    g = W.make_geometry(40, 0.25, 3, 4, 9.0, 200, support_radius_mm=4.5, t_min_us=base.t_min_us)
    xs, ys, zs = g.node_coords_mm()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    ones = np.ones(g.vol_shape)
    aff = 0.7 * X - 1.3 * Y + 2.1 * Z + 0.4
    g1 = oracle.G(g, ones)
    ga = oracle.G(g, aff)
    checked = 0
    for q in range(g.n_transducers):
        for k in range(0, g.n_samples, 7):
            P, _, _ = oracle.shell_points(g, q, k)
            n = len(P)
            assert g1[q, k] == pytest.approx(g.spacing_mm ** 2 * n, rel=1e-12, abs=0)
            want = g.spacing_mm ** 2 * (0.7 * P[:, 0] - 1.3 * P[:, 1] + 2.1 * P[:, 2] + 0.4).sum()
            assert ga[q, k] == pytest.approx(want, rel=1e-10, abs=1e-10)
            checked += n > 0
    assert checked > 20


def test_rotation_about_z_shifts_views():
    """P-symmetry: a centred square grid rotated by 90 degrees about z maps transducer
    (ring, view) to (ring, view + N_v/4); the local frames rotate with it, so the data
    move by N_v/4 views to rounding."""
    g = W.make_geometry((20, 20, 16), 0.3, 3, 8, 9.0, 120)
    a = W.spheres_phantom(g, 5, seed=21).astype(np.float64)
    n = g.nx
    # alpha'(R r) = alpha(r), R(x, y) = (-y, x): node (ix, iy) -> (n-1-iy, ix)
    rot = np.empty_like(a)
    for iy in range(n):
        for ix in range(n):
            rot[:, ix, n - 1 - iy] = a[:, iy, ix]
    d0 = oracle.G(g, a).reshape(3, 8, -1)
    d1 = oracle.G(g, rot).reshape(3, 8, -1)
    assert _rel(np.roll(d0, 2, axis=1), d1) < 1e-11


# ------------------------------------------------------------------------------------ closed form

def _sphere_case(ds):
    rs, a, amp = 10.0, 1.2, 1.0
    centre = np.array([0.3, -0.2, 0.25])
    n = int(math.ceil(2 * (a + 0.6) / ds)) + 1
    g = W.make_geometry(n, ds, 2, 3, rs, 128, fs_mhz=40.0, c=1.5)
    alpha = W.supersampled_sphere(g, centre, a, amp, ss=4)
    return g, alpha, centre, a, amp


@pytest.mark.parametrize("ds_pair", [(0.2, 0.1)])
def test_closed_form_uniform_sphere_srt(ds_pair):
    """P-closed: the discrete SRT of a partial-volume sphere approaches the exact SRT of a
    uniform sphere, g(t) = pi A c t (a^2 - (d - c t)^2) / d for |d - c t| <= a (Eq. srt), and
    the error decreases when the spacing is halved."""
    errs = []
    for ds in ds_pair:
        g, alpha, centre, a, amp = _sphere_case(ds)
        got = oracle.G(g, alpha)
        t = g.t_min_us + np.arange(g.n_samples) / g.fs_mhz
        rho = g.c_mm_per_us * t
        want = np.zeros_like(got)
        for q in range(g.n_transducers):
            d = np.linalg.norm(g.positions_mm[q] - centre)
            inside = np.abs(d - rho) <= a
            want[q, inside] = math.pi * amp * rho[inside] * (a * a - (d - rho[inside]) ** 2) / d
        errs.append(_rel(got, want))
    assert errs[0] < 0.05, errs
    assert errs[1] < errs[0], errs


def test_closed_form_uniform_sphere_pressure():
    """D G of the sphere approaches the N-shaped pulse p = (Gamma/2) A (d - c t)/d
    (Eqs. srt and g2p) away from the two edges of the pulse."""
    g, alpha, centre, a, amp = _sphere_case(0.1)
    g.gruneisen = 2.0
    p = oracle.H(g, alpha)
    t = g.t_min_us + np.arange(g.n_samples) / g.fs_mhz
    rho = g.c_mm_per_us * t
    for q in range(g.n_transducers):
        d = np.linalg.norm(g.positions_mm[q] - centre)
        core = np.abs(d - rho) <= a - 0.35
        want = 0.5 * g.gruneisen * amp * (d - rho[core]) / d
        assert core.sum() > 10
        assert _rel(p[q, core], want) < 0.05


# ------------------------------------------------------------------------------------ helpers

def test_pruned_node_gather_equals_full_scatter():
    """oracle.Gt_nodes (the only pruned routine) equals the full scatter at sampled nodes."""
    g = W.make_geometry(24, 0.25, 4, 4, 8.0, 96)
    y = W.random_data(g, seed=8).astype(np.float64)
    full = oracle.Gt(g, y)
    rng = np.random.default_rng(1)
    nodes = np.stack([rng.integers(0, g.nx, 40), rng.integers(0, g.ny, 40), rng.integers(0, g.nz, 40)], 1)
    nodes[0] = (0, 0, 0)
    nodes[1] = (g.nx - 1, g.ny - 1, g.nz - 1)
    got = oracle.Gt_nodes(g, y, nodes)
    want = full[nodes[:, 2], nodes[:, 1], nodes[:, 0]]
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(full).max())


def test_H_rows_equal_full_H():
    g = W.make_geometry(16, 0.3, 2, 3, 7.0, 64)
    a = W.spheres_phantom(g, 3, seed=2)
    full = oracle.H(g, a)
    rows = [(0, 0), (0, 1), (1, 30), (5, 63), (3, 20), (2, 62)]
    got = oracle.H_rows(g, a, rows)
    want = np.array([full[q, k] for q, k in rows])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-14)


def test_workload_reproduces_paper_scan():
    """The scanner generator reproduces the printed geometry of the simulation study."""
    with open(os.path.join(HERE, "golden", "paper_scan.json")) as f:
        ref = json.load(f)
    pos = W.arc_positions(ref["rings"], ref["views"], ref["measurement_radius_mm"])
    assert pos.shape == (ref["rings"] * ref["views"], 3)
    r = np.linalg.norm(pos, axis=1)
    assert np.allclose(r, ref["measurement_radius_mm"])
    th = np.arccos(pos[:, 2] / r)
    assert th.min() == pytest.approx(ref["theta_min_rad_times_256_over_pi"] * math.pi / 256)
    assert th.max() == pytest.approx(math.pi - math.pi / 256)
    cub = [n * ref["spacing_mm"] for n in ref["grid"]]
    assert np.allclose(cub, ref["cuboid_mm"])
