"""FP64 reference of the reconstruction layer (test infrastructure only).

Penalised least squares with a total-variation penalty and non-negativity,

    min_{x >= 0}  1/2 || H x - u ||^2 + mu TV(x),

which is the PLS objective of Sec. IV.A (Eq. PLSObjFuncInt) with TV in place of the quadratic
smoothness penalty of Sec. IV.B, solved by FISTA -- the fast-converging algorithm the paper's
Sec. V points to -- with the TV proximal map computed by the fast gradient projection on the
dual problem (Beck and Teboulle, 2009).  The steps are written in the order of those algorithms,
in double precision, with numpy primitives and no blocking or reordering.

TV(x) = sum_n || (x_{n+e_x} - x_n, x_{n+e_y} - x_n, x_{n+e_z} - x_n) ||_2, forward differences,
zero difference across the far boundary of each axis.  Volumes are (nz, ny, nx).
"""
from __future__ import annotations

import math

import numpy as np


def grad(x):
    """Forward differences (gx, gy, gz), zero on the last index of each axis."""
    gx = np.zeros_like(x); gy = np.zeros_like(x); gz = np.zeros_like(x)
    gx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    gy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    gz[:-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    return gx, gy, gz


def grad_t(px, py, pz):
    """Adjoint of grad: <grad x, p> = <x, grad_t p>."""
    out = np.zeros_like(px)
    # x-direction: d/dx_n of sum (x_{n+1} - x_n) p_n over n < N-1
    out[:, :, 1:] += px[:, :, :-1]
    out[:, :, :-1] -= px[:, :, :-1]
    out[:, 1:, :] += py[:, :-1, :]
    out[:, :-1, :] -= py[:, :-1, :]
    out[1:, :, :] += pz[:-1, :, :]
    out[:-1, :, :] -= pz[:-1, :, :]
    return out


def tv(x):
    gx, gy, gz = grad(np.asarray(x, np.float64))
    return float(np.sqrt(gx * gx + gy * gy + gz * gz).sum())


def tv_prox(z, lam, iters, g=None, step=0.0):
    """argmin_{x >= 0} 1/2 ||x - z'||^2 + lam TV(x), z' = z - step g, by `iters` iterations of FGP:
    x(r) = max(0, z' - lam grad^T r); p <- Proj_{|.|<=1}(r + grad x(r) / (12 lam)) (12 bounds
    ||grad||^2 in 3-D); r <- p + (t_k - 1)/t_{k+1} (p - p_prev); final x(p)."""
    z = np.asarray(z, np.float64)
    if g is not None:
        z = z - step * np.asarray(g, np.float64)
    if lam == 0.0 or iters == 0:
        return np.maximum(z, 0.0)
    p = [np.zeros_like(z) for _ in range(3)]
    r = [np.zeros_like(z) for _ in range(3)]
    t = 1.0
    for _ in range(iters):
        x = np.maximum(z - lam * grad_t(*r), 0.0)
        gx, gy, gz = grad(x)
        a = r[0] + gx / (12.0 * lam)
        b = r[1] + gy / (12.0 * lam)
        c = r[2] + gz / (12.0 * lam)
        nrm = np.maximum(1.0, np.sqrt(a * a + b * b + c * c))
        pn = [a / nrm, b / nrm, c / nrm]
        tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        mom = (t - 1.0) / tn
        r = [pn[i] + mom * (pn[i] - p[i]) for i in range(3)]
        p = pn
        t = tn
    return np.maximum(z - lam * grad_t(*p), 0.0)


def fista_tv(H, Ht, u, mu, L, iters, x0, inner=10):
    """FISTA on 1/2||Hx - u||^2 + mu TV(x), x >= 0, step 1/L (L >= ||H||^2).  Iterates
    x_k = prox_{(mu/L) TV + [x>=0]}(y_k - H^T(H y_k - u)/L), t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
    y_{k+1} = x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1}).  Returns the iterates' relative data
    residuals ||H x_k - u|| / ||u|| and the final x."""
    u = np.asarray(u, np.float64)
    x_prev = np.asarray(x0, np.float64).copy()
    y = x_prev.copy()
    t = 1.0
    res = []
    un = np.linalg.norm(u)
    for _ in range(iters):
        gradf = Ht(H(y) - u)
        x = tv_prox(y, mu / L, inner, g=gradf, step=1.0 / L)
        res.append(float(np.linalg.norm(H(x) - u) / un))
        tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        y = x + ((t - 1.0) / tn) * (x - x_prev)
        x_prev = x
        t = tn
    return x_prev, res
