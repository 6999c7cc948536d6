"""FP64 reference of the spherical-voxel imaging model H_sph and its adjoint (test infrastructure
only: the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it).

Sec. II.B (Eqs. basissph, coeffsph, dis_sph, p0f, ddmodelsp) models the object as uniform spheres
of diameter Delta_s at the grid nodes r_n and the data as temporal-frequency samples of the
pressure at each transducer,

    [u~]_{qL+l} = p~0(f_l) sum_n alpha_n h~_q(r_n, f_l) / S_q,

and for point transducers h~_q(r_n, f) / S_q is the integrand of the SIR at the transducer,
exp(-j 2 pi f |r_q - r_n| / c) / (2 pi |r_q - r_n|).  Eq. p0f gives the spectrum of one voxel's
pulse,

    p~0(f) = -j (beta c^3 / (C_p f)) [ Delta_s / (2 c) cos(pi f Delta_s / c)
                                       - sin(pi f Delta_s / c) / (2 pi f) ] h~e(f),

with beta c^2 / C_p = Gamma.  The adjoint (Eq. sphbwd) for a real coefficient vector and the real
inner product Re <u, v> is

    [H_sph^T u~]_n = Re sum_q sum_l u~_{qL+l} conj(p~0(f_l)) conj(h~_q(r_n, f_l) / S_q).

Readings taken here:
  - alpha_n is the mean of A over the n-th spherical voxel (Eq. coeffsph's prefactor read so that
    a uniform object of value A gives alpha_n = A; this is what makes dis_sph reproduce the
    pressure pulse of a uniform sphere, the pin in tests/test_sph_oracle.py);
  - the frequencies are any list f_l > 0 (the paper's data are L = 511 components in (0, 5] MHz,
    f_l = (l + 1) Delta_f); the transducer response h~e(f_l) is an optional complex array
    (1 for the simulation studies);
  - Fourier convention P(f) = int p(t) exp(-j 2 pi f t) dt (the sign of Eq. dis_sph's phase).

Written as the plain sums, one transducer at a time, vectorised over voxels and frequencies with
numpy in double precision.
"""
from __future__ import annotations

import math

import numpy as np


def p0_tilde(freqs_mhz, spacing_mm, c_mm_per_us, gruneisen=1.0, eir=None):
    """p~0(f_l) of Eq. p0f (complex, one per frequency)."""
    f = np.asarray(freqs_mhz, np.float64)
    ds, c = float(spacing_mm), float(c_mm_per_us)
    x = math.pi * f * ds / c
    val = -1j * (gruneisen * c / f) * (ds / (2.0 * c) * np.cos(x) - np.sin(x) / (2.0 * math.pi * f))
    if eir is not None:
        val = val * np.asarray(eir, np.complex128)
    return val


def _nodes(geom):
    xs, ys, zs = geom.node_coords_mm()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def H_sph(geom, alpha, freqs_mhz, eir=None, qs=None):
    """u~ [Q][L] (complex) = H_sph alpha for alpha (nz, ny, nx) (Eq. dis_sph); qs selects
    transducers (rows) only."""
    a = np.asarray(alpha, np.float64).ravel()
    f = np.asarray(freqs_mhz, np.float64)
    p0 = p0_tilde(f, geom.spacing_mm, geom.c_mm_per_us, geom.gruneisen, eir)
    rn = _nodes(geom)
    qs = range(geom.n_transducers) if qs is None else qs
    out = np.zeros((len(qs), len(f)), np.complex128)
    for r, q in enumerate(qs):
        d = np.linalg.norm(rn - geom.positions_mm[q], axis=1)
        for l in range(len(f)):
            h = np.exp(-2j * math.pi * f[l] * d / geom.c_mm_per_us) / (2.0 * math.pi * d)
            out[r, l] = p0[l] * np.dot(h, a)
    return out


def H_sph_t(geom, u, freqs_mhz, eir=None, nodes=None):
    """alpha' = H_sph^T u~ for u~ [Q][L] (complex) (Eq. sphbwd): the whole grid (nz, ny, nx), or
    the nodes given as (ix, iy, iz) triples (a 1-D array)."""
    u = np.asarray(u, np.complex128).reshape(geom.n_transducers, -1)
    f = np.asarray(freqs_mhz, np.float64)
    p0 = p0_tilde(f, geom.spacing_mm, geom.c_mm_per_us, geom.gruneisen, eir)
    if nodes is None:
        rn = _nodes(geom)
    else:
        xs, ys, zs = geom.node_coords_mm()
        nd = np.asarray(nodes, np.int64).reshape(-1, 3)
        rn = np.stack([xs[nd[:, 0]], ys[nd[:, 1]], zs[nd[:, 2]]], axis=1)
    out = np.zeros(len(rn))
    w = u * np.conj(p0)[None, :]                                  # u~_{q,l} conj(p~0(f_l))
    for q in range(geom.n_transducers):
        d = np.linalg.norm(rn - geom.positions_mm[q], axis=1)
        for c0 in range(0, len(rn), 4096):                        # nodes in chunks, all frequencies at once
            dc = d[c0:c0 + 4096]
            hc = np.exp(2j * math.pi * f[:, None] * dc[None, :] / geom.c_mm_per_us) / (2.0 * math.pi * dc[None, :])
            out[c0:c0 + 4096] += (w[q] @ hc).real
    return out.reshape(geom.vol_shape) if nodes is None else out
