"""Pins of the FP64 U-Net reference against library routines.  CPU only."""
import numpy as np
from scipy import ndimage

from oracle import unet


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((6, 7, 5, 3))
    w = rng.standard_normal((27, 4, 3))
    got = unet.conv3d(x, w)
    for co in range(4):
        want = np.zeros(x.shape[:3])
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3, 3)      # [dz][dy][dx]
            want += ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        assert np.allclose(got[..., co], want, atol=1e-12)


def test_pool_and_upsample_are_adjoint_shaped():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 8, 2))
    y = rng.standard_normal((2, 3, 4, 2))
    # <avgpool2 x, y> = <x, upsample2(y) / 8>
    assert np.isclose((unet.avgpool2(x) * y).sum(), (x * unet.upsample2(y) / 8).sum())
    assert unet.forward(unet.init_params(0), rng.standard_normal((8, 8, 8))).shape == (8, 8, 8)


def test_forward_matches_a_torch_nn_unet():
    """The composition of oracle/unet.py's forward against the same network built from torch.nn
    modules in FP64, written from the architecture alone: three levels of two 3x3x3 'same'
    convolutions with ReLU (16, 32, 64 channels), 2x2x2 average pooling between levels, nearest
    2x upsampling on the way up, concatenated in front of the skip connection of the level, and a
    1x1x1 head; the single input channel feeds the first convolution.  Weights and (non-zero)
    biases are copied over.  A change of the skip order, the pooling or upsampling placement, the
    head or the input channel fails this."""
    import pytest
    torch = pytest.importorskip("torch")
    import torch.nn as nn
    import torch.nn.functional as Fn

    p = unet.init_params(3)
    rng = np.random.default_rng(4)
    for name, cin, cout in unet.LAYERS:
        p[name + ".b"] = 0.1 * rng.standard_normal(cout)
    p["head.b"] = 0.3

    def conv(cin, cout, name, first=False):
        m = nn.Conv3d(cin, cout, 3, padding=1).double()
        w = p[name + ".w"]                                     # [tap][cout][cin], tap = (dz 3 + dy) 3 + dx
        w = w[:, :, :1] if first else w
        with torch.no_grad():
            m.weight.copy_(torch.from_numpy(np.ascontiguousarray(w.transpose(1, 2, 0))).reshape(cout, cin, 3, 3, 3))
            m.bias.copy_(torch.from_numpy(p[name + ".b"]))
        return m

    class Net(nn.Module):
        def __init__(self):
            super().__init__()
            self.e1 = nn.ModuleList([conv(1, 16, "e1a", first=True), conv(16, 16, "e1b")])
            self.e2 = nn.ModuleList([conv(16, 32, "e2a"), conv(32, 32, "e2b")])
            self.b = nn.ModuleList([conv(32, 64, "b1"), conv(64, 64, "b2")])
            self.d2 = nn.ModuleList([conv(96, 32, "d2a"), conv(32, 32, "d2b")])
            self.d1 = nn.ModuleList([conv(48, 16, "d1a"), conv(16, 16, "d1b")])
            self.head = nn.Conv3d(16, 1, 1).double()
            with torch.no_grad():
                self.head.weight.copy_(torch.from_numpy(p["head.w"]).reshape(1, 16, 1, 1, 1))
                self.head.bias.fill_(p["head.b"])

        @staticmethod
        def block(mods, x):
            for m in mods:
                x = torch.relu(m(x))
            return x

        def forward(self, x):
            s1 = self.block(self.e1, x)
            s2 = self.block(self.e2, Fn.avg_pool3d(s1, 2))
            bt = self.block(self.b, Fn.avg_pool3d(s2, 2))
            d2 = self.block(self.d2, torch.cat([Fn.interpolate(bt, scale_factor=2, mode="nearest"), s2], dim=1))
            d1 = self.block(self.d1, torch.cat([Fn.interpolate(d2, scale_factor=2, mode="nearest"), s1], dim=1))
            return self.head(d1)

    inp = rng.standard_normal((12, 8, 16))
    want = Net()(torch.from_numpy(inp)[None, None]).detach().numpy()[0, 0]
    got = unet.forward(p, inp)
    assert got.shape == inp.shape
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), np.abs(got - want).max()
