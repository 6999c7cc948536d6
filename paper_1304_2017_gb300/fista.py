"""FISTA-TV reconstruction on the device.

Solves  min_{x >= 0} 1/2 ||H x - u||^2 + mu TV(x)  -- the penalised least-squares objective of
Sec. IV.A (Eq. PLSObjFuncInt) with a total-variation penalty -- by FISTA (Beck and Teboulle,
2009; the paper's Sec. V names fast-converging algorithms as the route to fewer iterations).
Every step runs in liboat.so: H and H^T (oat_project / oat_backproject), the TV proximal map with
the gradient step fused in (oat_tv_prox), the momentum and residual updates, and the FP64
reductions.  This module only orders the calls and reads back two FP64 scalars per iteration
(the relative data residual and the stopping test).

By linearity H y_{k+1} = (1 + beta_k) H x_k - beta_k H x_{k-1}, so one iteration costs one H and
one H^T and yields the exact residual ||H x_k - u|| of the iterate.
"""
from __future__ import annotations

import math
import time

import torch

from . import oat


class FistaTV:
    def __init__(self, plan, mu, L=None, inner=10):
        self.plan = plan
        self.mu = float(mu)
        self.inner = int(inner)
        self.L = L
        dev = torch.device("cuda", plan.device)
        nz, ny, nx = plan.vol_shape
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.M = plan.data_shape[0] * plan.data_shape[1]
        f = dict(dtype=torch.float32, device=dev)
        self.x = torch.zeros(plan.vol_shape, **f)
        self.x_prev = torch.zeros(plan.vol_shape, **f)
        self.y = torch.zeros(plan.vol_shape, **f)
        self.g = torch.zeros(plan.vol_shape, **f)
        self.work = torch.zeros(7 * self.N, **f)
        self.hx = torch.zeros(plan.data_shape, **f)
        self.hx_prev = torch.zeros(plan.data_shape, **f)
        self.r = torch.zeros(plan.data_shape, **f)
        self.acc = torch.zeros(4, dtype=torch.float64, device=dev)

    def _s(self):
        return torch.cuda.current_stream(self.plan.device).cuda_stream

    def lipschitz(self, iters=30, seed=0, safety=1.02):
        """Largest eigenvalue of H^T H by power iteration (FP64 norms), times a safety factor."""
        gen = torch.Generator(device=self.x.device).manual_seed(seed)
        v = torch.rand(self.plan.vol_shape, generator=gen, device=self.x.device)
        lam = 0.0
        for _ in range(iters):
            self.acc.zero_()
            oat.oat_dot(self.N, v.data_ptr(), v.data_ptr(), self.acc.data_ptr(), self._s())
            nv = math.sqrt(float(self.acc[0]))
            v.mul_(1.0 / nv)
            w = self.plan.backproject(self.plan.project(v))
            self.acc.zero_()
            oat.oat_dot(self.N, v.data_ptr(), w.data_ptr(), self.acc.data_ptr(), self._s())
            lam = float(self.acc[0])
            v = w
        self.L = lam * safety
        return self.L

    def solve(self, u, iters, tol=None, x0=None, callback=None):
        """Run up to `iters` iterations from x0 (zeros if None).  u: the measured data, float32,
        float16 or bfloat16 (read exactly; the iteration itself runs in float32 on a float32
        plan).  Returns (x, info) with the relative data residuals of the iterates and the
        cumulative GPU time (CUDA events)."""
        if self.L is None:
            self.lipschitz()
        plan, s = self.plan, self._s()
        L, lam = float(self.L), self.mu / float(self.L)
        nx, ny, nz = self.shape
        if x0 is None:
            self.x_prev.zero_()
        else:
            self.x_prev.copy_(x0)
        self.y.copy_(self.x_prev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        plan.project(self.x_prev, out=self.hx_prev)
        self.acc.zero_()
        ud = oat.dtype_code(u.dtype)
        oat.oat_fista_residual(self.M, self.hx_prev.data_ptr(), self.hx_prev.data_ptr(), u.data_ptr(), ud, 0.0,
                               self.r.data_ptr(), self.acc.data_ptr(), s)
        res0 = math.sqrt(float(self.acc[0]) / max(float(self.acc[1]), 1e-300))
        t = 1.0
        history, times = [], []
        for k in range(iters):
            plan.backproject(self.r, out=self.g)                                    # H^T (H y_k - u)
            oat.oat_tv_prox(nx, ny, nz, self.y.data_ptr(), self.g.data_ptr(), 1.0 / L, lam, self.inner,
                            self.x.data_ptr(), self.work.data_ptr(), s)           # x_k
            plan.project(self.x, out=self.hx)                                      # H x_k
            tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            beta = (t - 1.0) / tn
            self.acc.zero_()
            oat.oat_fista_residual(self.M, self.hx.data_ptr(), self.hx_prev.data_ptr(), u.data_ptr(), ud, beta,
                                   self.r.data_ptr(), self.acc.data_ptr(), s)     # r = H y_{k+1} - u
            oat.oat_fista_momentum(self.N, self.x.data_ptr(), self.x_prev.data_ptr(), beta, self.y.data_ptr(), s)
            self.x, self.x_prev = self.x_prev, self.x
            self.hx, self.hx_prev = self.hx_prev, self.hx
            t = tn
            ev1.record()
            res = math.sqrt(float(self.acc[0]) / max(float(self.acc[1]), 1e-300))  # synchronises
            history.append(res)
            times.append(ev0.elapsed_time(ev1) * 1e-3)
            if callback is not None:
                callback(k, res)
            if tol is not None and res <= tol:
                break
        return self.x_prev, {"residual": history, "gpu_seconds": times, "residual0": res0, "L": L}
