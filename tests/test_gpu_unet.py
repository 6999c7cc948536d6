"""The U-Net kernels (BF16 convolutions on the 5th-generation tensor cores, backward kernels)
against the FP64 reference (oracle/unet.py).  BF16 storage bounds the agreement: outputs are rounded to 8-bit
mantissas (relative 2^-9), so elementwise comparisons use 2^-8 of the reference magnitude."""
import ctypes

import numpy as np
import pytest

from oracle import unet as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1304_2017_gb300 import unet
    return torch, unet


def bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("cin,cout,shape", [(16, 16, (5, 7, 9)), (32, 64, (4, 6, 70)), (48, 16, (3, 5, 17)),
                                            (64, 96, (4, 4, 8))])
def test_conv3d_forward_and_input_gradient(env, cin, cout, shape):
    torch, unet = env
    rng = np.random.default_rng(cin + cout)
    x = bf16_round(rng.standard_normal(shape + (cin,)))
    w = bf16_round(rng.standard_normal((27, cout, cin)) * 0.1)
    b = rng.standard_normal(cout).astype(np.float32)
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    wt = torch.from_numpy(w.astype(np.float32)).cuda().to(torch.bfloat16)
    bt = torch.from_numpy(b).cuda()
    y = torch.empty(shape + (cout,), dtype=torch.bfloat16, device="cuda")
    z, yy, xx = shape
    unet._call("oat_conv3d_bf16", xx, yy, z, cin, cout, unet._p(xt), unet._p(wt), unet._p(bt), 1, unet._p(y), None)
    torch.cuda.synchronize()
    unet._call("oat_unet_check")          # no pipeline wait of the tensor-core kernel ran out
    want = ref.conv3d(x, w, b.astype(np.float64), relu=True)
    got = y.float().cpu().numpy()
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-6 * np.abs(want).max())
    # input gradient: same kernel, weights flipped in space and transposed in channels
    if cin in (16, 32, 48, 64, 96):
        g = bf16_round(rng.standard_normal(shape + (cout,)))
        gt = torch.from_numpy(g.astype(np.float32)).cuda().to(torch.bfloat16)
        wf = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
        dx = torch.empty(shape + (cin,), dtype=torch.bfloat16, device="cuda")
        unet._call("oat_conv3d_flip_weights", cin, cout, unet._p(wt), unet._p(wf), None)
        if cout % 16 == 0:
            unet._call("oat_conv3d_bf16", xx, yy, z, cout, cin, unet._p(gt), unet._p(wf), None, 0, unet._p(dx), None)
            torch.cuda.synchronize()
            unet._call("oat_unet_check")
            # adjoint: <conv(x, w), g> = <x, conv^T(g)>; conv^T written out from the definition
            wflip = np.transpose(w[::-1], (0, 2, 1))
            want_dx = ref.conv3d(g, wflip)
            got_dx = dx.float().cpu().numpy()
            assert np.all(np.abs(got_dx - want_dx) <= 2.0 ** -8 * np.abs(want_dx) + 1e-6 * np.abs(want_dx).max())
            lhs = (ref.conv3d(x, w) * g).sum()
            assert lhs == pytest.approx((x * want_dx).sum(), rel=1e-9)


@pytest.mark.parametrize("shape", [(8, 16, 128), (4, 6, 200), (2, 3, 1)])
def test_conv3d_tile_shapes(env, shape):
    """Tiles of 128 voxels along x (one row), several tiles per row with a partial last one, and a
    row of one voxel: the tensor-core kernel against the FP64 convolution."""
    torch, unet = env
    rng = np.random.default_rng(sum(shape))
    cin, cout = 32, 48
    x = bf16_round(rng.standard_normal(shape + (cin,)))
    w = bf16_round(rng.standard_normal((27, cout, cin)) * 0.1)
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    wt = torch.from_numpy(w.astype(np.float32)).cuda().to(torch.bfloat16)
    y = torch.empty(shape + (cout,), dtype=torch.bfloat16, device="cuda")
    z, yy, xx = shape
    unet._call("oat_conv3d_bf16", xx, yy, z, cin, cout, unet._p(xt), unet._p(wt), None, 0, unet._p(y), None)
    torch.cuda.synchronize()
    unet._call("oat_unet_check")
    want = ref.conv3d(x, w)
    got = y.float().cpu().numpy()
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-6 * np.abs(want).max())


def test_conv3d_rejects_unaligned(env):
    """The TMA copies and vector stores need 16-byte alignment: refused on the host."""
    torch, unet = env
    from paper_1304_2017_gb300 import oat
    x = torch.zeros(4 * 4 * 4 * 16 + 8, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(27 * 16 * 16, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(4 * 4 * 4 * 16, dtype=torch.bfloat16, device="cuda")
    rc = unet._lib.oat_conv3d_bf16(4, 4, 4, 16, 16, ctypes.c_void_p(x.data_ptr() + 2), unet._p(w), None, 0,
                                   unet._p(y), None)
    assert rc == oat.OAT_ERR_INVALID_ARG and "aligned" in oat.oat_last_error()


def test_weight_gradient(env):
    torch, unet = env
    rng = np.random.default_rng(3)
    shape, cin, cout = (6, 7, 9), 32, 16
    x = bf16_round(rng.standard_normal(shape + (cin,)))
    g = bf16_round(rng.standard_normal(shape + (cout,)))
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    gt = torch.from_numpy(g.astype(np.float32)).cuda().to(torch.bfloat16)
    dw = torch.zeros(27 * cout * cin, device="cuda")
    db = torch.zeros(cout, device="cuda")
    z, y, xx = shape
    unet._call("oat_conv3d_wgrad", xx, y, z, cin, cout, unet._p(xt), unet._p(gt), unet._p(dw), unet._p(db), None)
    torch.cuda.synchronize()
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    want = np.zeros((27, cout, cin))
    for tap in range(27):
        dz, dy, dx_ = tap // 9, (tap // 3) % 3, tap % 3
        want[tap] = np.einsum("zyxo,zyxi->oi", g, xp[dz:dz + z, dy:dy + y, dx_:dx_ + xx])
    assert np.allclose(dw.cpu().numpy().reshape(27, cout, cin), want, rtol=1e-4, atol=1e-4)
    assert np.allclose(db.cpu().numpy(), g.sum(axis=(0, 1, 2)), rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("shape,cin,cout", [((6, 10, 200), 32, 16), ((3, 4, 5), 96, 32), ((2, 2, 130), 16, 64)])
def test_weight_gradient_tiles_and_determinism(env, shape, cin, cout):
    """Weight and bias gradients on the tensor cores over several x tiles, voxel splits and channel
    counts, against the FP64 sum; two calls give bit-identical results (fixed-order reduction)."""
    torch, unet = env
    rng = np.random.default_rng(sum(shape) + cin)
    x = bf16_round(rng.standard_normal(shape + (cin,)))
    g = bf16_round(rng.standard_normal(shape + (cout,)))
    xt = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    gt = torch.from_numpy(g.astype(np.float32)).cuda().to(torch.bfloat16)
    z, y, xx = shape
    outs = []
    for _ in range(2):
        dw = torch.zeros(27 * cout * cin, device="cuda")
        db = torch.zeros(cout, device="cuda")
        unet._call("oat_conv3d_wgrad", xx, y, z, cin, cout, unet._p(xt), unet._p(gt), unet._p(dw), unet._p(db), None)
        torch.cuda.synchronize()
        unet._call("oat_unet_check")
        outs.append((dw.clone(), db.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    want = np.zeros((27, cout, cin))
    for tap in range(27):
        dz, dy, dx_ = tap // 9, (tap // 3) % 3, tap % 3
        want[tap] = np.einsum("zyxo,zyxi->oi", g, xp[dz:dz + z, dy:dy + y, dx_:dx_ + xx])
    got = outs[0][0].cpu().numpy().reshape(27, cout, cin)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-5 * scale, np.abs(got - want).max() / scale
    assert np.allclose(outs[0][1].cpu().numpy(), g.sum(axis=(0, 1, 2)), rtol=1e-5, atol=1e-5 * np.abs(g).sum(axis=(0, 1, 2)).max())


def test_network_gradient_against_fp64_finite_differences(env):
    """Loss = mean (net(x) - t)^2 on an 8^3 grid: parameter gradients of the device backward
    (BF16 activations) against central differences of the FP64 reference network with the same
    BF16-rounded weights."""
    torch, unet = env
    rng = np.random.default_rng(4)
    params = ref.init_params(7)
    for name, _, _ in ref.LAYERS:
        params[name + ".w"] = bf16_round(params[name + ".w"])
        params[name + ".b"] = rng.standard_normal(params[name + ".b"].shape) * 0.05
    inp = np.abs(rng.standard_normal((8, 8, 8)))
    inp = bf16_round(inp)
    target = rng.standard_normal((8, 8, 8)) * 0.5
    net = unet.UNet((8, 8, 8), params=params)
    vt = torch.from_numpy(inp.astype(np.float32)).cuda()
    tt = torch.from_numpy(target.astype(np.float32)).cuda()
    net.forward(vt, 1.0)
    net.zero_grad()
    net.backward(net.mse_grad(tt))
    torch.cuda.synchronize()
    out = net.out.cpu().numpy()
    want_out = ref.forward(params, inp)
    assert np.linalg.norm(out - want_out) <= 0.02 * np.linalg.norm(want_out)

    def loss(p):
        return ((ref.forward(p, inp) - target) ** 2).mean()

    picks = [("head.w", (3,)), ("head.b", ()), ("d1b.w", (13, 2, 5)), ("d2a.w", (4, 7, 70)), ("b2.w", (13, 11, 40)),
             ("e2a.w", (22, 9, 1)), ("e1a.w", (13, 4, 0)), ("e1b.b", (6,)), ("b1.b", (33,)), ("d1a.w", (0, 15, 40))]
    got, fd = [], []
    for key, idx in picks:
        h = 1e-3
        p_plus = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in params.items()}
        p_minus = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in params.items()}
        if key == "head.b":
            p_plus[key] += h; p_minus[key] -= h
        else:
            p_plus[key][idx] += h; p_minus[key][idx] -= h
        fd.append((loss(p_plus) - loss(p_minus)) / (2 * h))
        gk = net.g[key].cpu().numpy()
        got.append(float(gk[idx]) if key != "head.b" else float(gk[0]))
    got, fd = np.array(got), np.array(fd)
    assert np.linalg.norm(got - fd) <= 0.05 * np.linalg.norm(fd), (got, fd)


def test_training_reduces_loss(env):
    torch, unet = env
    rng = np.random.default_rng(5)
    net = unet.UNet((16, 16, 16), seed=1)
    inp = torch.from_numpy(np.abs(rng.standard_normal((16, 16, 16))).astype(np.float32)).cuda()
    tgt = torch.from_numpy((0.5 * np.abs(rng.standard_normal((16, 16, 16)))).astype(np.float32)).cuda()
    losses = []
    for _ in range(60):
        net.forward(inp, 1.0)
        net.zero_grad()
        net.backward(net.mse_grad(tgt))
        losses.append(float(net.loss[0]))
        net.adam(lr=3e-3)
    assert losses[-1] < 0.5 * losses[0], losses[::10]
