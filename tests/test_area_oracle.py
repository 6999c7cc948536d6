"""Pins of the exact-area variant of the shell lattice (point weight Delta_s 2 pi rho
sin(theta_i) / N_j, the area of ring i's strip of the shell shared by its N_j points) in the FP64
oracle, against geometry recomputed from the points themselves, a closed-form sum, the
Appendix's uniform weights and the closed-form SRT of a uniform sphere (Eq. srt).  CPU only."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1304_2017_gb300 import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _area(g):
    return dataclasses.replace(g, lattice_weights=1)


def _shells(g):
    """A few shells per transducer: near the front of the object, the middle and the back."""
    K = g.n_samples
    return [(q, k) for q in range(g.n_transducers) for k in (K // 3, K // 2, 2 * K // 3)]


def test_ring_weights_from_point_geometry():
    """Every ring's weights sum to Delta_s 2 pi rho sin(theta), with rho and theta measured from
    the ring's points (distance to the transducer, angle to the inward axis), and are equal
    within the ring; the Appendix's weights are Delta_s^2 for every point."""
    g = W.make_geometry(24, 0.25, 2, 3, 7.0, 90)
    ga = _area(g)
    ds = g.spacing_mm
    checked = 0
    for q, k in _shells(g):
        P, ij, nr, w = oracle.shell_points(ga, q, k, with_weights=True)
        _, _, _, wu = oracle.shell_points(g, q, k, with_weights=True)
        assert np.all(wu == ds * ds)
        if len(P) == 0:
            continue
        rq = g.positions_mm[q]
        ez = -rq / np.linalg.norm(rq)
        v = P - rq
        rho = np.linalg.norm(v, axis=1)
        cos_t = (v @ ez) / rho
        for i in np.unique(ij[:, 0]):
            m = ij[:, 0] == i
            sin_t = math.sqrt(max(0.0, 1.0 - float(np.mean(cos_t[m])) ** 2))
            want = ds * 2.0 * math.pi * float(np.mean(rho[m])) * sin_t
            assert abs(w[m].sum() - want) <= 1e-10 * want
            assert np.ptp(w[m]) <= 1e-14 * w[m].max()
            checked += 1
    assert checked > 50


def test_shell_total_closed_form_and_floor_bias():
    """Over a shell the weights total Delta_s 2 pi rho sum_{i<N} sin(i dtheta), which has the
    closed form sin(N dtheta / 2) sin((N - 1) dtheta / 2) / sin(dtheta / 2); the Appendix's
    weights fall short of it by the rounding of 2 pi / dphi_i down to N_j (at most one point
    per ring)."""
    g = W.make_geometry(24, 0.25, 2, 3, 7.0, 90)
    ga = _area(g)
    ds = g.spacing_mm
    for q, k in _shells(g):
        P, ij, nr, w = oracle.shell_points(ga, q, k, with_weights=True)
        if nr < 2:
            continue
        rho = g.c_mm_per_us * (g.t_min_us + k / g.fs_mhz)
        dth = ds / rho
        want = ds * 2 * math.pi * rho * math.sin(nr * dth / 2) * math.sin((nr - 1) * dth / 2) / math.sin(dth / 2)
        assert abs(w.sum() - want) <= 1e-11 * want
        uniform = len(P) * ds * ds
        assert uniform <= w.sum() * (1 + 1e-12)
        assert w.sum() - uniform <= nr * ds * ds


def test_area_weights_tighten_the_uniform_sphere_srt():
    """The discrete SRT of a partial-volume sphere against the exact SRT of a uniform sphere,
    g(t) = pi A c t (a^2 - (d - c t)^2) / d (Eq. srt): exact strip areas come closer than the
    Appendix's weights, and closer still when the spacing is halved."""
    rs, a, amp = 10.0, 1.2, 1.0
    centre = np.array([0.3, -0.2, 0.25])
    errs = {}
    for ds in (0.2, 0.1):
        n = int(math.ceil(2 * (a + 0.6) / ds)) + 1
        g = W.make_geometry(n, ds, 2, 3, rs, 128, fs_mhz=40.0, c=1.5)
        alpha = W.supersampled_sphere(g, centre, a, amp, ss=4)
        t = g.t_min_us + np.arange(g.n_samples) / g.fs_mhz
        rho = g.c_mm_per_us * t
        want = np.zeros(g.data_shape)
        for q in range(g.n_transducers):
            d = np.linalg.norm(g.positions_mm[q] - centre)
            inside = np.abs(d - rho) <= a
            want[q, inside] = math.pi * amp * rho[inside] * (a * a - (d - rho[inside]) ** 2) / d
        for lw in (0, 1):
            errs[(ds, lw)] = _rel(oracle.G(dataclasses.replace(g, lattice_weights=lw), alpha), want)
    print(errs)
    assert errs[(0.2, 1)] < errs[(0.2, 0)] and errs[(0.1, 1)] < errs[(0.1, 0)], errs
    assert errs[(0.1, 1)] < errs[(0.2, 1)], errs


def test_area_dense_and_adjoint():
    """With exact strip areas the oracle's G still equals the dense matrix assembled from
    psi_n's definition, G^T its transpose (full scatter and pruned node gather), and D G / G^T D^T
    stay adjoint."""
    g = _area(W.config("tiny"))
    M = oracle.dense_G(g)
    x = W.random_volume(g, seed=3).astype(np.float64)
    y = W.random_data(g, seed=4).astype(np.float64)
    assert _rel(oracle.G(g, x).ravel(), M @ x.ravel()) < 1e-12
    gty = oracle.Gt(g, y)
    assert _rel(gty.ravel(), M.T @ y.ravel()) < 1e-12
    nodes = np.array([[i, j, l] for i in range(g.nx) for j in range(g.ny) for l in range(g.nz)])
    assert _rel(oracle.Gt_nodes(g, y, nodes), gty[nodes[:, 2], nodes[:, 1], nodes[:, 0]]) < 1e-12
    # a weight really differs from Delta_s^2 here
    assert _rel(M, oracle.dense_G(dataclasses.replace(g, lattice_weights=0))) > 1e-3
    lhs = float((oracle.H(g, x) * y).sum())
    rhs = float((x * oracle.Ht(g, y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-300
