"""Pins of the FP64 FBP reference (oracle/fbp.py, Eq. disfbp) against facts other than itself.

1. Data linear in time, p = a + b t: the linear interpolation and the first difference are then
   exact, so the discrete formula must equal the continuous integrand of Eq. fbp,
   [2 p / t + dp/dt] at t = |r - r_q| / c, summed with the patch weights -- to rounding.  This
   fixes the sign, the prefactor, the 1.5 factors and the t_min offsets.
2. A uniform sphere: its exact pressure (the N-shaped pulse p = (Gamma/2) A (d - c t) / d for
   |d - c t| <= a, Eqs. srt and g2p) sampled in time and reconstructed by FBP gives back the
   amplitude A inside the sphere (Finch's formula is exact in 3-D); the error decreases when the
   temporal and angular sampling are refined.  (Outside the sphere the jumps of the pulse leave
   shell-shaped streaks whose size depends on the ratio of angular to temporal sampling; only
   the interior is pinned.)
"""
import math

import numpy as np
import pytest

from oracle import fbp as F
from paper_1304_2017_gb300 import workloads as W


def test_linear_data_matches_continuous_integrand():
    g = W.make_geometry((7, 6, 5), 0.5, 4, 6, 12.0, 400, fs_mhz=20.0, t_min_us=4.0)
    a, b = 0.7, -0.3
    dt = 1.0 / g.fs_mhz
    t = g.t_min_us + dt * np.arange(g.n_samples)
    p = np.tile(a + b * t, (g.n_transducers, 1))
    w = F.arc_weights(g.positions_mm, 4, 6)
    got = F.fbp(g, p, w)
    xs, ys, zs = g.node_coords_mm()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    want = np.zeros(g.vol_shape)
    for q in range(g.n_transducers):
        rq = g.positions_mm[q]
        tq = np.sqrt((X - rq[0]) ** 2 + (Y - rq[1]) ** 2 + (Z - rq[2]) ** 2) / g.c_mm_per_us
        assert tq.min() >= t[0] and tq.max() <= t[-2]            # every sample pair inside the window
        want += w[q] * (2.0 * (a + b * tq) / tq + b)
    want *= -1.0 / (2.0 * math.pi * g.gruneisen * g.c_mm_per_us)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def _sphere_fbp(n_rings, n_views, fs, amp=0.8, a=2.0):
    g = W.make_geometry(13, 0.4, n_rings, n_views, 12.0, int(12 * fs), fs_mhz=fs, t_min_us=2.0)
    c = g.c_mm_per_us
    dt = 1.0 / fs
    t = g.t_min_us + dt * np.arange(g.n_samples)
    d = np.linalg.norm(g.positions_mm, axis=1)[:, None]        # sphere at the origin
    ct = c * t[None, :]
    p = np.where(np.abs(d - ct) <= a, 0.5 * g.gruneisen * amp * (d - ct) / d, 0.0)
    rec = F.fbp(g, p, F.arc_weights(g.positions_mm, n_rings, n_views))
    xs, ys, zs = g.node_coords_mm()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    inner = rec[r <= 0.5 * a]
    return abs(inner.mean() - amp) / amp, float(np.abs(inner - amp).max() / amp)


def test_uniform_sphere_reconstructs_its_amplitude():
    mean_coarse, max_coarse = _sphere_fbp(16, 32, 20.0)
    mean_fine, max_fine = _sphere_fbp(32, 64, 40.0)
    assert mean_coarse < 0.005 and max_coarse < 0.02, (mean_coarse, max_coarse)
    assert mean_fine < 0.5 * mean_coarse and max_fine < max_coarse, (mean_fine, max_fine)


def test_out_of_window_samples_are_zero():
    g = W.make_geometry(6, 0.5, 2, 3, 8.0, 40, t_min_us=1.0)
    p = np.zeros(g.data_shape)
    # samples that no node reaches (far before the first arrival) contribute nothing
    p[:, :3] = 1.0
    assert np.abs(F.fbp(g, p, np.ones(g.n_transducers))).max() == 0.0


def test_sample_positions_at_known_distances():
    """sample_positions (Eq. linearint's k~) at nodes whose distance to the transducer is known:
    a transducer on the z axis and nodes on that axis, with t_min chosen so that node 0 sits
    exactly on sample 37 and each further node (one spacing closer) 0.27 / (c dt) samples earlier."""
    g = W.make_geometry(9, 0.27, 1, 1, 6.0, 200, positions_mm=[[0.0, 0.0, 6.0]])
    dt = 1.0 / g.fs_mhz
    xs, ys, zs = g.node_coords_mm()
    ix = int(np.argmin(np.abs(xs)))
    iy = int(np.argmin(np.abs(ys)))
    assert xs[ix] == 0.0 and ys[iy] == 0.0                 # odd node count: a node column on the axis
    d0 = 6.0 - zs[0]
    g.t_min_us = d0 / g.c_mm_per_us - 37 * dt
    nodes = np.array([[ix, iy, iz] for iz in range(g.nz)])
    kt = F.sample_positions(g, nodes, np.zeros(g.nz, int))
    want = 37.0 - np.arange(g.nz) * 0.27 / (g.c_mm_per_us * dt)
    assert np.allclose(kt, want, rtol=0, atol=1e-10), np.abs(kt - want).max()
