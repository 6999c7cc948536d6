"""FP64 reference of the filtered backprojection (test infrastructure only).

The continuous FBP formula for a spherical measurement surface S of radius R^s (Sec. II, Eq. fbp,
after Finch et al.) reconstructs

    A(r) = -C_p / (2 pi beta c^3 R^s) * int_S dS [ 2 p(r^s, t) / t + dp/dt (r^s, t) ],
           t = |r - r^s| / c,

and its discretisation (Sec. III.C, Eqs. linearint and disfbp) approximates
  - the surface integral by patches of area (R^s)^2 dtheta dphi sin(theta_q),
  - p(t) by linear interpolation between the samples k and k + 1 around
    k~ = (|r_q - r_n| / c - t_min) / dt (k the integer part of k~),
  - dp/dt by (p_{k+1} - p_k) / dt,
which gives, with tau0 = t_min / dt and C_p / beta = c^2 / Gamma,

    alpha_n = -1 / (pi Gamma c dt) * sum_q w_q { (1.5 - (k + tau0) / (k~ + tau0)) p_{q,k+1}
                                              + ((k + 1 + tau0) / (k~ + tau0) - 1.5) p_{q,k} },
    w_q = R^s dtheta dphi sin(theta_q)   (patch area / R^s).

Readings taken here:
  - the weights w_q are an input (one per transducer), so that any transducer layout can be
    described; for the rings x views scan of Sec. III.A, w_q = R^s (pi / N_r)(2 pi / N_v)
    sin(theta_q) (`arc_weights`);
  - samples outside 0 .. K-1 count as zero (no extrapolation);
  - p is the data vector itself (point transducers: the measured data are the pressure).

Written in the order of Eq. disfbp, one transducer at a time, vectorised over the nodes with
numpy in double precision.
"""
from __future__ import annotations

import math

import numpy as np


def arc_weights(positions_mm, n_rings, n_views):
    """w_q = R^s dtheta dphi sin(theta_q) for the scan of Sec. III.A (rings x views, dtheta =
    pi / N_r, dphi = 2 pi / N_v); theta_q is the polar angle of transducer q."""
    pos = np.asarray(positions_mm, np.float64)
    rs = np.linalg.norm(pos, axis=1)
    theta = np.arccos(np.clip(pos[:, 2] / rs, -1.0, 1.0))
    return rs * (math.pi / n_rings) * (2.0 * math.pi / n_views) * np.sin(theta)


def sample_positions(geom, nodes, transducers):
    """k~ = (|r_q - r_n| / c - t_min) / dt (Eq. linearint) in FP64 for (node, transducer) pairs:
    nodes (n, 3) integer (ix, iy, iz), transducers (n,) integer."""
    nd = np.asarray(nodes, np.int64).reshape(-1, 3)
    qs = np.asarray(transducers, np.int64).reshape(-1)
    o = np.asarray(geom.origin_mm, np.float64)
    r = o[None, :] + geom.spacing_mm * nd.astype(np.float64)
    d = np.sqrt(((r - geom.positions_mm[qs]) ** 2).sum(axis=1))
    return (d / geom.c_mm_per_us - geom.t_min_us) / (1.0 / geom.fs_mhz)


def fbp(geom, p, weights, nodes=None, absolute=False):
    """alpha_fbp from data p [Q][K] (Eq. disfbp): on the whole node grid of `geom` as
    (nz, ny, nx), or at the nodes given as (ix, iy, iz) triples (a 1-D array).

    absolute=True sums the terms' magnitudes instead (the scale of the sum's rounding)."""
    p = np.asarray(p, np.float64).reshape(geom.data_shape)
    w = np.asarray(weights, np.float64).reshape(geom.n_transducers)
    dt = 1.0 / geom.fs_mhz
    c = geom.c_mm_per_us
    tau0 = geom.t_min_us / dt
    K = geom.n_samples
    xs, ys, zs = geom.node_coords_mm()
    if nodes is None:
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    else:
        nd = np.asarray(nodes, np.int64).reshape(-1, 3)
        X, Y, Z = xs[nd[:, 0]], ys[nd[:, 1]], zs[nd[:, 2]]
    acc = np.zeros(X.shape)

    def term(q, k, kt):
        def sample(j):
            inside = (j >= 0) & (j < K)
            return np.where(inside, p[q, np.clip(j, 0, K - 1)], 0.0)
        pk, pk1 = sample(k), sample(k + 1)
        tau = kt + tau0
        return w[q] * ((1.5 - (k + tau0) / tau) * pk1 + ((k + 1 + tau0) / tau - 1.5) * pk)

    for q in range(geom.n_transducers):
        rq = geom.positions_mm[q]
        dist = np.sqrt((X - rq[0]) ** 2 + (Y - rq[1]) ** 2 + (Z - rq[2]) ** 2)
        kt = (dist / c - geom.t_min_us) / dt                 # k~
        k = np.floor(kt).astype(np.int64)
        t = term(q, k, kt)
        acc += np.abs(t) if absolute else t
    scale = 1.0 / (math.pi * geom.gruneisen * c * dt)
    return (1.0 if absolute else -1.0) * acc * scale
