"""Learned warm start for PLS-TV: a 3-level 3-D U-Net (16 / 32 / 64 channels) on the device.

The network maps the backprojection H^T y (scaled by its maximum) to an initial estimate x_0
for FISTA-TV.  Convolutions run in liboat.so's tensor-core kernels (BF16 activations and
weights, FP32 accumulation in tensor memory, tcgen05.mma, include/oat_unet.h); training uses the library's own backward
kernels (input gradients by the same convolution with flipped weights, weight gradients on the
FP32 cores) and an Adam step kernel.  This module orders the calls and owns the buffers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import oat

LAYERS = [("e1a", 16, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("b1", 32, 64), ("b2", 64, 64),
          ("d2a", 96, 32), ("d2b", 32, 32), ("d1a", 48, 16), ("d1b", 16, 16)]

_lib = oat.lib
_vp, _i, _ll, _f = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_float
_SIGS = {
    "oat_conv3d_bf16": [_i, _i, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp],
    "oat_conv3d_flip_weights": [_i, _i, _vp, _vp, _vp],
    "oat_conv3d_wgrad": [_i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp],
    "oat_add_bf16": [_ll, _vp, _vp, _vp, _vp],
    "oat_relu_grad": [_ll, _vp, _vp, _vp, _vp],
    "oat_avgpool2": [_i, _i, _i, _i, _vp, _vp, _i, _vp],
    "oat_upsample2": [_i, _i, _i, _i, _vp, _i, _i, _vp, _i, _vp],
    "oat_copy_channels": [_ll, _i, _vp, _i, _i, _vp, _i, _i, _vp],
    "oat_pack_input": [_ll, _vp, _f, _vp, _vp],
    "oat_head": [_ll, _i, _vp, _vp, _vp, _vp, _vp],
    "oat_head_grad": [_ll, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "oat_mse": [_ll, _vp, _vp, _vp, _vp, _vp],
    "oat_adam": [_ll, _vp, _vp, _vp, _vp, _f, _f, _f, _f, _i, _vp, _vp],
    "oat_unet_check": [],
}
for _n, _a in _SIGS.items():
    getattr(_lib, _n).argtypes = _a
    getattr(_lib, _n).restype = ctypes.c_int


def _call(name, *args):
    rc = getattr(_lib, name)(*args)
    if rc != 0:
        raise oat.OatError(rc, oat.oat_last_error())


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class UNet:
    """Buffers and parameters for one grid size (nz, ny, nx), each divisible by 4."""

    def __init__(self, shape, device=0, seed=0, params=None):
        nz, ny, nx = shape
        assert nz % 4 == 0 and ny % 4 == 0 and nx % 4 == 0, "grid sizes must be multiples of 4"
        self.shape = shape
        self.dev = torch.device("cuda", device)
        if params is None:
            from_np = _init_params(seed)
        else:
            from_np = params
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.p, self.pb, self.g, self.m, self.v = {}, {}, {}, {}, {}
        for name, _, _ in LAYERS:
            for suf in (".w", ".b"):
                key = name + suf
                self.p[key] = torch.tensor(np.asarray(from_np[key], np.float32), **f32).contiguous()
        self.p["head.w"] = torch.tensor(np.asarray(from_np["head.w"], np.float32), **f32)
        self.p["head.b"] = torch.tensor(np.asarray([from_np["head.b"]], np.float32), **f32).reshape(1)
        for k, t in self.p.items():
            self.g[k] = torch.zeros_like(t)
            self.m[k] = torch.zeros_like(t)
            self.v[k] = torch.zeros_like(t)
            if k.endswith(".w") and not k.startswith("head"):
                self.pb[k] = t.to(torch.bfloat16).contiguous()
        self.step_count = 0
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        s1, s2, s4 = shape, tuple(d // 2 for d in shape), tuple(d // 4 for d in shape)
        self.sizes = {1: s1, 2: s2, 4: s4}
        A = {}
        for key, lv, c in (("x16", 1, 16), ("e1a", 1, 16), ("e1b", 1, 16), ("p1", 2, 16), ("e2a", 2, 32), ("e2b", 2, 32),
                           ("p2", 4, 32), ("b1", 4, 64), ("b2", 4, 64), ("cat2", 2, 96), ("d2a", 2, 32), ("d2b", 2, 32),
                           ("cat1", 1, 48), ("d1a", 1, 16), ("d1b", 1, 16)):
            A[key] = torch.zeros(self.sizes[lv] + (c,), **bf)
        self.a = A
        self.G = {k: torch.zeros_like(t) for k, t in A.items()}     # gradients of the activations
        self.tmp = {lv: torch.zeros(self.sizes[lv] + (96,), **bf) for lv in (1, 2, 4)}
        self.out = torch.zeros(shape, **f32)
        self.dout = torch.zeros(shape, **f32)
        self.loss = torch.zeros(2, dtype=torch.float64, device=self.dev)
        self.wf = {name: torch.zeros(27 * cin * cout, **bf) for name, cin, cout in LAYERS}

    def _s(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream)

    def nvox(self, lv):
        z, y, x = self.sizes[lv]
        return z * y * x

    def _conv(self, name, lv, x, y, relu=True):
        cin, cout = dict((n, (a, b)) for n, a, b in LAYERS)[name]
        z, yy, xx = self.sizes[lv]
        _call("oat_conv3d_bf16", xx, yy, z, cin, cout, _p(x), _p(self.pb[name + ".w"]), _p(self.p[name + ".b"]),
              1 if relu else 0, _p(y), self._s())

    def forward(self, vol, scale):
        """vol: (nz, ny, nx) float32 on the device; returns the (nz, ny, nx) float32 estimate."""
        s, a = self._s(), self.a
        z, y, x = self.sizes[1]
        _call("oat_pack_input", self.nvox(1), _p(vol), ctypes.c_float(scale), _p(a["x16"]), s)
        self._conv("e1a", 1, a["x16"], a["e1a"])
        self._conv("e1b", 1, a["e1a"], a["e1b"])
        _call("oat_avgpool2", x, y, z, 16, _p(a["e1b"]), _p(a["p1"]), 0, s)
        self._conv("e2a", 2, a["p1"], a["e2a"])
        self._conv("e2b", 2, a["e2a"], a["e2b"])
        z2, y2, x2 = self.sizes[2]
        _call("oat_avgpool2", x2, y2, z2, 32, _p(a["e2b"]), _p(a["p2"]), 0, s)
        self._conv("b1", 4, a["p2"], a["b1"])
        self._conv("b2", 4, a["b1"], a["b2"])
        z4, y4, x4 = self.sizes[4]
        _call("oat_upsample2", x4, y4, z4, 64, _p(a["b2"]), 96, 0, _p(a["cat2"]), 0, s)
        _call("oat_copy_channels", self.nvox(2), 32, _p(a["e2b"]), 32, 0, _p(a["cat2"]), 96, 64, s)
        self._conv("d2a", 2, a["cat2"], a["d2a"])
        self._conv("d2b", 2, a["d2a"], a["d2b"])
        _call("oat_upsample2", x2, y2, z2, 32, _p(a["d2b"]), 48, 0, _p(a["cat1"]), 0, s)
        _call("oat_copy_channels", self.nvox(1), 16, _p(a["e1b"]), 16, 0, _p(a["cat1"]), 48, 32, s)
        self._conv("d1a", 1, a["cat1"], a["d1a"])
        self._conv("d1b", 1, a["d1a"], a["d1b"])
        _call("oat_head", self.nvox(1), 16, _p(a["d1b"]), _p(self.p["head.w"]), _p(self.p["head.b"]), _p(self.out), s)
        return self.out

    def _back_conv(self, name, lv, x_in, y_out, g_out, g_in):
        """Gradient through y = relu(conv(x)): weight/bias grads, and the input gradient into
        g_in (skipped when g_in is None)."""
        s = self._s()
        cin, cout = dict((n, (a, b)) for n, a, b in LAYERS)[name]
        z, yy, xx = self.sizes[lv]
        gpre = self.tmp[lv].view(-1)[: self.nvox(lv) * cout]   # [voxel][cout] pre-activation gradient
        _call("oat_relu_grad", self.nvox(lv) * cout, _p(y_out), _p(g_out), _p(gpre), s)
        _call("oat_conv3d_wgrad", xx, yy, z, cin, cout, _p(x_in), _p(gpre), _p(self.g[name + ".w"]),
              _p(self.g[name + ".b"]), s)
        if g_in is not None:
            _call("oat_conv3d_flip_weights", cin, cout, _p(self.pb[name + ".w"]), _p(self.wf[name]), s)
            _call("oat_conv3d_bf16", xx, yy, z, cout, cin, _p(gpre), _p(self.wf[name]), None, 0, _p(g_in), s)

    def backward(self, dout):
        """Gradients of all parameters for the output gradient dout (float32, accumulated)."""
        s, a, G = self._s(), self.a, self.G
        z, y, x = self.sizes[1]
        z2, y2, x2 = self.sizes[2]
        z4, y4, x4 = self.sizes[4]
        _call("oat_head_grad", self.nvox(1), 16, _p(a["d1b"]), _p(self.p["head.w"]), _p(dout), _p(G["d1b"]),
              _p(self.g["head.w"]), _p(self.g["head.b"]), s)
        self._back_conv("d1b", 1, a["d1a"], a["d1b"], G["d1b"], G["d1a"])
        self._back_conv("d1a", 1, a["cat1"], a["d1a"], G["d1a"], G["cat1"])
        _call("oat_upsample2", x2, y2, z2, 32, _p(G["cat1"]), 48, 0, _p(G["d2b"]), 1, s)
        self._back_conv("d2b", 2, a["d2a"], a["d2b"], G["d2b"], G["d2a"])
        self._back_conv("d2a", 2, a["cat2"], a["d2a"], G["d2a"], G["cat2"])
        _call("oat_upsample2", x4, y4, z4, 64, _p(G["cat2"]), 96, 0, _p(G["b2"]), 1, s)
        self._back_conv("b2", 4, a["b1"], a["b2"], G["b2"], G["b1"])
        self._back_conv("b1", 4, a["p2"], a["b1"], G["b1"], G["p2"])
        # e2b receives the pooled path and the skip connection
        _call("oat_avgpool2", x2, y2, z2, 32, _p(G["p2"]), _p(G["e2b"]), 1, s)
        _call("oat_copy_channels", self.nvox(2), 32, _p(G["cat2"]), 96, 64, _p(G["e2a"]), 32, 0, s)
        _call("oat_add_bf16", self.nvox(2) * 32, _p(G["e2b"]), _p(G["e2a"]), _p(G["e2b"]), s)
        self._back_conv("e2b", 2, a["e2a"], a["e2b"], G["e2b"], G["e2a"])
        self._back_conv("e2a", 2, a["p1"], a["e2a"], G["e2a"], G["p1"])
        _call("oat_avgpool2", x, y, z, 16, _p(G["p1"]), _p(G["e1b"]), 1, s)
        _call("oat_copy_channels", self.nvox(1), 16, _p(G["cat1"]), 48, 32, _p(G["e1a"]), 16, 0, s)
        _call("oat_add_bf16", self.nvox(1) * 16, _p(G["e1b"]), _p(G["e1a"]), _p(G["e1b"]), s)
        self._back_conv("e1b", 1, a["e1a"], a["e1b"], G["e1b"], G["e1a"])
        self._back_conv("e1a", 1, a["x16"], a["e1a"], G["e1a"], None)

    def zero_grad(self):
        for t in self.g.values():
            t.zero_()

    def mse_grad(self, target):
        """loss = mean (out - target)^2 (FP64 on the device); self.dout receives its gradient."""
        self.loss.zero_()
        _call("oat_mse", self.out.numel(), _p(self.out), _p(target), _p(self.dout), _p(self.loss), self._s())
        return self.dout

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for k, t in self.p.items():
            _call("oat_adam", t.numel(), _p(t), _p(self.g[k]), _p(self.m[k]), _p(self.v[k]), ctypes.c_float(lr),
                  ctypes.c_float(b1), ctypes.c_float(b2), ctypes.c_float(eps), self.step_count, _p(self.pb.get(k)),
                  self._s())

    def state(self):
        return {k: t.detach().cpu().numpy().astype(np.float64) for k, t in self.p.items()}


def _init_params(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))
        p[name + ".b"] = np.zeros(cout)
    p["head.w"] = rng.standard_normal(16) * np.sqrt(1.0 / 16)
    p["head.b"] = 0.0
    return p
