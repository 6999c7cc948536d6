"""The transducer response as numpy convolutions, row by row: the identity the FP64 reference
(oracle/eir.py) is pinned to, used where a record is too long for its explicit sums."""
import numpy as np


def conv_rows(p, h, m0):
    """H^e p row by row as numpy's full linear convolution shifted by 1 + m0 samples (the
    identity the reference is pinned to), for records too long for its explicit sums."""
    K = p.shape[1]
    out = np.zeros_like(p)
    for q in range(p.shape[0]):
        full = np.convolve(p[q], h)                       # full[t] = sum_i h_i p_{t-i}
        for k in range(K):
            t = k - 1 - m0
            if 0 <= t < len(full):
                out[q, k] = full[t]
    return out


def corr_rows(u, h, m0):
    """H^e^T u row by row: p'_k = sum_i h_i u_{k+1+m0+i} = full(u, reversed h)[k + m0 + n]."""
    K, n = u.shape[1], len(h)
    out = np.zeros_like(u)
    for q in range(u.shape[0]):
        full = np.convolve(u[q], h[::-1])
        for k in range(K):
            t = k + m0 + n
            if 0 <= t < len(full):
                out[q, k] = full[t]
    return out
