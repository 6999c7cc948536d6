"""FP64 reference of the transducer response H^e and its adjoint (test infrastructure only).

Sec. II.B (Eq. EIR): the measured data are the pressure convolved in time with the transducer's
acousto-electric impulse response, discretised as

    [H^e p]_{q,k} = sum_{kappa=0}^{K-1} h_{k-1-kappa} p_{q,kappa},

with h_m = dt h^e(m dt); and the adjoint (Sec. II.B, "Adjoints of the system matrices")

    [H^e^T u]_{q,k} = sum_{kappa=0}^{K-1} h_{kappa-1-k} u_{q,kappa}.

The full model is H = H^e D G and its adjoint G^T D^T H^e^T.

Reading: the taps are given as an array h of n values for m = m0, m0 + 1, ..., m0 + n - 1
(h_m = 0 outside), so that causal (m0 >= 0) and centred responses are both described; sums run
over the window 0 .. K-1 only, as the formula states.  Written as the explicit sums, in the order
of the formulas, one transducer row at a time.
"""
from __future__ import annotations

import numpy as np


def _tap(h, m0, m):
    j = m - m0
    return h[j] if 0 <= j < len(h) else 0.0


def Heir(p, h, m0=0):
    """u = H^e p for data p [Q][K] (Eq. EIR)."""
    p = np.asarray(p, np.float64)
    h = np.asarray(h, np.float64)
    Q, K = p.shape
    u = np.zeros((Q, K))
    for k in range(K):
        for kappa in range(K):
            c = _tap(h, m0, k - 1 - kappa)
            if c != 0.0:
                u[:, k] += c * p[:, kappa]
    return u


def Heir_t(u, h, m0=0):
    """p' = H^e^T u for data u [Q][K]."""
    u = np.asarray(u, np.float64)
    h = np.asarray(h, np.float64)
    Q, K = u.shape
    p = np.zeros((Q, K))
    for k in range(K):
        for kappa in range(K):
            c = _tap(h, m0, kappa - 1 - k)
            if c != 0.0:
                p[:, k] += c * u[:, kappa]
    return p
