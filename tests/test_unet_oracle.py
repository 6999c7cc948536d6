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
