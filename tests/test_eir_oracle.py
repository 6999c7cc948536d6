"""Pins of the FP64 transducer-response reference (oracle/eir.py, Eq. EIR) against facts other
than itself: special kernels whose action is known, numpy's linear convolution, and the
adjoint identity."""
import numpy as np

from oracle import eir as E
from eir_conv import conv_rows, corr_rows


def test_identity_and_delay_kernels():
    rng = np.random.default_rng(1)
    p = rng.standard_normal((3, 17))
    # h_{-1} = 1: u_k = p_k (the formula's one-sample offset cancels)
    assert np.array_equal(E.Heir(p, [1.0], m0=-1), p)
    # h_0 = 1: a delay by one sample, the first sample falls out of the window
    u = E.Heir(p, [1.0], m0=0)
    assert np.array_equal(u[:, 1:], p[:, :-1]) and np.all(u[:, 0] == 0.0)
    # h_{-3} = 2: an advance by two samples, scaled
    u = E.Heir(p, [2.0], m0=-3)
    assert np.array_equal(u[:, :-2], 2.0 * p[:, 2:]) and np.all(u[:, -2:] == 0.0)


def test_matches_numpy_convolution():
    """u_k = sum_m h_m p_{k-1-m} is numpy's full linear convolution of p with h, shifted by
    1 + m0 samples and cut to the window."""
    rng = np.random.default_rng(2)
    p = rng.standard_normal((4, 40))
    h = rng.standard_normal(9)
    for m0 in (-4, 0, 3):
        u = E.Heir(p, h, m0=m0)
        for q in range(p.shape[0]):
            full = np.convolve(p[q], h)                  # full[n] = sum_j h_j p_{n-j}
            shift = 1 + m0                               # u_k = full[k - shift]
            want = np.array([full[k - shift] if 0 <= k - shift < len(full) else 0.0 for k in range(40)])
            assert np.allclose(u[q], want, rtol=1e-13, atol=1e-13)


def test_adjoint_identity():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((5, 31))
    u = rng.standard_normal((5, 31))
    h = rng.standard_normal(7)
    for m0 in (-3, 0, 2):
        lhs = float((E.Heir(p, h, m0) * u).sum())
        rhs = float((p * E.Heir_t(u, h, m0)).sum())
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(p) * np.linalg.norm(u)


def test_long_record_helpers_match_the_reference():
    """The convolution helpers of the long-record test equal the reference on a short record."""
    rng = np.random.default_rng(9)
    p = rng.standard_normal((2, 50)); h = rng.standard_normal(13)
    for m0 in (-20, -7, 0, 4):
        assert np.allclose(conv_rows(p, h, m0), E.Heir(p, h, m0), rtol=1e-12, atol=1e-12)
        assert np.allclose(corr_rows(p, h, m0), E.Heir_t(p, h, m0), rtol=1e-12, atol=1e-12)
