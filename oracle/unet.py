"""FP64 reference of the learned warm start's network (test infrastructure only).

A 3-level 3-D U-Net (16 / 32 / 64 channels): two 3x3x3 'same' convolutions with ReLU per level,
2x2x2 average pooling down, nearest 2x upsampling and channel concatenation up, a 1x1x1 head.
Tensors are (z, y, x, c); weights w[tap][cout][cin], tap = (dz * 3 + dy) * 3 + dx for offsets
(dz - 1, dy - 1, dx - 1).  Written from the definition of the convolution (a sum over the 27
taps), in double precision.
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout) of the 3x3x3 convolutions, in forward order
LAYERS = [("e1a", 16, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("b1", 32, 64), ("b2", 64, 64),
          ("d2a", 96, 32), ("d2b", 32, 32), ("d1a", 48, 16), ("d1b", 16, 16)]


def conv3d(x, w, b=None, relu=False):
    Z, Y, X, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((Z, Y, X, w.shape[1]))
    for tap in range(27):
        dz, dy, dx = tap // 9, (tap // 3) % 3, tap % 3
        out += xp[dz:dz + Z, dy:dy + Y, dx:dx + X, :] @ w[tap].T
    if b is not None:
        out += b
    return np.maximum(out, 0.0) if relu else out


def avgpool2(x):
    Z, Y, X, C = x.shape
    return x.reshape(Z // 2, 2, Y // 2, 2, X // 2, 2, C).mean(axis=(1, 3, 5))


def upsample2(x):
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def forward(params, inp):
    """inp: (z, y, x) float volume (already scaled); returns the (z, y, x) output."""
    x = np.zeros(inp.shape + (16,))
    x[..., 0] = inp
    c = lambda name, v: conv3d(v, params[name + ".w"], params[name + ".b"], relu=True)  # noqa: E731
    s1 = c("e1b", c("e1a", x))
    s2 = c("e2b", c("e2a", avgpool2(s1)))
    bt = c("b2", c("b1", avgpool2(s2)))
    d2 = c("d2b", c("d2a", np.concatenate([upsample2(bt), s2], axis=-1)))
    d1 = c("d1b", c("d1a", np.concatenate([upsample2(d2), s1], axis=-1)))
    return d1 @ params["head.w"] + params["head.b"]


def init_params(seed=0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".w"] = rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))
        p[name + ".b"] = np.zeros(cout)
    p["head.w"] = rng.standard_normal(16) * np.sqrt(1.0 / 16)
    p["head.b"] = 0.0
    return p
