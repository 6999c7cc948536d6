"""Pins of the FP64 spherical-voxel reference (oracle/sph.py, Eqs. dis_sph, p0f, sphbwd) against
facts other than itself: the Fourier transform, taken by numerical quadrature, of the pressure
pulse of a uniform sphere (Eqs. srt and g2p: p = (Gamma / 2) A (d - c t) / d for |d - c t| <= a),
the zero-frequency limit of Eq. p0f, and the adjoint identity.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import sph as S
from paper_1304_2017_gb300 import workloads as W


def _pulse_spectrum(f, d, a, amp, gamma, c):
    """P(f) = int p(t) exp(-j 2 pi f t) dt of the N-shaped pulse of a uniform sphere of radius a
    and value amp at distance d, by adaptive quadrature."""
    p = lambda t: 0.5 * gamma * amp * (d - c * t) / d
    t0, t1 = (d - a) / c, (d + a) / c
    w = 2 * math.pi * f
    re = integrate.quad(p, t0, t1, weight="cos", wvar=w, epsabs=0, epsrel=1e-10)[0]
    im = -integrate.quad(p, t0, t1, weight="sin", wvar=w, epsabs=0, epsrel=1e-10)[0]
    return re + 1j * im


@pytest.mark.parametrize("gamma", [1.0, 2.5])
def test_single_voxel_is_the_uniform_sphere_pulse(gamma):
    """A single spherical voxel (diameter Delta_s, value A) seen by a point transducer: H_sph
    gives the spectrum of the sphere's N-shaped pulse at every frequency."""
    ds, c = 0.3, 1.5
    geom = W.make_geometry(5, ds, 1, 3, 6.0, 16, c=c, gruneisen=gamma)
    alpha = np.zeros(geom.vol_shape)
    alpha[2, 1, 3] = 0.8                                   # node (ix, iy, iz) = (3, 1, 2)
    freqs = np.array([0.05, 0.7, 1.9, 3.3, 5.0])
    u = S.H_sph(geom, alpha, freqs)
    xs, ys, zs = geom.node_coords_mm()
    rn = np.array([xs[3], ys[1], zs[2]])
    for q in range(geom.n_transducers):
        d = float(np.linalg.norm(geom.positions_mm[q] - rn))
        for l, f in enumerate(freqs):
            want = _pulse_spectrum(f, d, ds / 2, 0.8, gamma, c)
            assert abs(u[q, l] - want) <= 1e-9 * abs(want) + 1e-15, (q, f, u[q, l], want)


def test_p0_vanishes_at_zero_frequency():
    """The bracket of Eq. p0f is -(Delta_s / 2c)(pi f Delta_s / c)^2 / 3 + O(f^4), so p~0(f) -> 0
    linearly: p~0(f) / f -> j Gamma c (Delta_s / 2c)(pi Delta_s / c)^2 / 3."""
    ds, c, g = 0.2, 1.5, 1.7
    f = np.array([1e-3, 1e-4])
    want = 1j * g * c * (ds / (2 * c)) * (math.pi * ds / c) ** 2 / 3
    got = S.p0_tilde(f, ds, c, g) / f
    assert np.allclose(got, want, rtol=1e-5)


def test_eir_multiplies_each_frequency():
    ds, c = 0.25, 1.5
    geom = W.make_geometry(4, ds, 1, 2, 5.0, 8, c=c)
    rng = np.random.default_rng(2)
    alpha = rng.standard_normal(geom.vol_shape)
    freqs = np.linspace(0.2, 4.0, 7)
    eir = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    assert np.allclose(S.H_sph(geom, alpha, freqs, eir=eir), S.H_sph(geom, alpha, freqs) * eir[None, :],
                       rtol=1e-13, atol=0)


def test_adjoint_identity():
    """Re <H_sph alpha, u> = <alpha, H_sph^T u> (real coefficients, complex data)."""
    geom = W.make_geometry((5, 4, 6), 0.3, 2, 3, 6.0, 8)
    rng = np.random.default_rng(3)
    alpha = rng.standard_normal(geom.vol_shape)
    freqs = (np.arange(9) + 1) * 0.5
    eir = np.exp(1j * rng.uniform(0, 2 * math.pi, 9))
    u = rng.standard_normal((geom.n_transducers, 9)) + 1j * rng.standard_normal((geom.n_transducers, 9))
    lhs = float(np.real(np.vdot(S.H_sph(geom, alpha, freqs, eir=eir), u)))
    rhs = float((alpha * S.H_sph_t(geom, u, freqs, eir=eir)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    # node subset equals the grid
    nodes = np.array([[1, 2, 3], [4, 0, 5], [0, 3, 0]])
    full = S.H_sph_t(geom, u, freqs, eir=eir)
    assert np.allclose(S.H_sph_t(geom, u, freqs, eir=eir, nodes=nodes), full[nodes[:, 2], nodes[:, 1], nodes[:, 0]],
                       rtol=1e-13, atol=0)
