"""Parity of the sm_103a filtered backprojection (oat_fbp, through the C ABI) with the FP64
reference oracle/fbp.py (Eq. disfbp).

Tolerance 1e-5 relative L2, on the raw difference: per term the kernel keeps the sample position
to about 1e-6 of a sample (float-pair distance to each brick centre, small FP32 offsets) and sums
with compensation, so its error stays near FP32 rounding of the data and weights.  FP16 / BF16
data are read exactly, so the reference gets the same rounded values.

Eq. disfbp is discontinuous in the sample position: where k~ crosses an integer the one-sided
difference p_{k+1} - p_k moves to the next pair.  The kernel therefore recomputes k~ in double
precision wherever its FP32 value lies within a guard band of an integer (half-width
g = 1e-5 (ds / (c dt) + 1) samples), so that it reads the pair the exact k~ selects.  The FP32
error of k~ is measured directly (oat_fbp_sample_positions against the FP64 definition) and must
stay below a quarter of g, which is what makes the band sufficient.  The forward-model cases
(smooth blobs and uniform spheres, whose pulses have sharp edges) are the ones with crossings
that move a node visibly."""
import numpy as np
import pytest

from oracle import fbp as F
from paper_1304_2017_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1304_2017_gb300 import oat
    return torch, oat


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# Half-width of the kernel's guard band in samples (fbp.cu, fbp_guard): 1e-5 grid units of
# distance plus 1e-5 samples.
def guard(geom):
    sk = geom.spacing_mm * geom.fs_mhz / geom.c_mm_per_us
    return 1e-5 * (sk + 1.0)


def smooth_data(geom, seed, width=6.0, n_pulses=3):
    """Per transducer, a sum of Gaussian pulses (width `width` samples) at seeded delays."""
    rng = np.random.default_rng(seed)
    k = np.arange(geom.n_samples)[None, :]
    p = np.zeros(geom.data_shape)
    for _ in range(n_pulses):
        c = rng.uniform(0, geom.n_samples, size=(geom.n_transducers, 1))
        a = rng.uniform(-1, 1, size=(geom.n_transducers, 1))
        p += a * np.exp(-0.5 * ((k - c) / width) ** 2)
    return p.astype(np.float32)


def blob_phantom(geom, seed, n=3, sigma_vox=2.5):
    """Sum of Gaussian blobs (standard deviation sigma_vox grid spacings): a smooth object, so
    that its data are band-limited."""
    rng = np.random.default_rng(seed)
    xs, ys, zs = geom.node_coords_mm()
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    s = sigma_vox * geom.spacing_mm
    vol = np.zeros(geom.vol_shape)
    for _ in range(n):
        c = [rng.uniform(v[len(v) // 4], v[3 * len(v) // 4]) for v in (xs, ys, zs)]
        vol += rng.uniform(0.3, 1.0) * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    return vol.astype(np.float32)


def _data(geom, kind, seed):
    if kind == "smooth":
        return smooth_data(geom, seed)
    if kind == "noise":
        # white N(0,1) data: the second difference at a crossing is as large as the data, so a
        # pair read on the wrong side of an integer would show at once
        return np.random.default_rng(seed).standard_normal(geom.data_shape).astype(np.float32)
    import oracle
    if kind == "spheres":
        # the forward model's own data (the oracle, FP64) of uniform spheres: sharp edges, so large
        # second differences where the pulses switch on and off
        return oracle.H(geom, W.spheres_phantom(geom, 3, seed=seed)).astype(np.float32)
    # the forward model's own data (the oracle, FP64) of a smooth object
    return oracle.H(geom, blob_phantom(geom, seed)).astype(np.float32)


CASES = {
    # non-round sizes: with round ones (0.3 mm, 9 mm, rings at multiples of 30 degrees) many
    # node-transducer distances land exactly on a sample, where Eq. disfbp switches its
    # difference pair and the reference's own rounding decides the side
    "ragged": (lambda: W.make_geometry((13, 10, 11), 0.31, 3, 5, 9.13, 120), "smooth"),
    "tmin0": (lambda: W.make_geometry(12, 0.29, 2, 4, 6.07, 120, t_min_us=0.0), "smooth"),
    "window_cut": (lambda: W.make_geometry(14, 0.31, 3, 4, 8.11, 30), "smooth"),
    "physical": (lambda: W.make_geometry(20, 0.251, 6, 8, 8.03, 160), "forward"),
    "physical_spheres": (lambda: W.make_geometry(20, 0.251, 6, 8, 8.03, 160), "spheres"),
    "physical_noise": (lambda: W.make_geometry(20, 0.251, 6, 8, 8.03, 160), "noise"),
    # coarse grid at 40 MHz: about 16 samples per grid spacing, so a brick's sample windows are
    # too wide to stage in shared memory and the kernel reads the data directly
    "coarse_direct": (lambda: W.make_geometry(10, 0.61, 3, 4, 9.13, 400, fs_mhz=40.0), "smooth"),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_fbp_matches_reference(env, case, dtype):
    torch, oat = env
    make, kind = CASES[case]
    geom = make()
    n_r = {"ragged": 3, "tmin0": 2, "window_cut": 3, "physical": 6, "physical_spheres": 6, "physical_noise": 6,
           "coarse_direct": 3}[case]
    n_v = geom.n_transducers // n_r
    w = F.arc_weights(geom.positions_mm, n_r, n_v)
    p = _data(geom, kind, 11)
    plan = oat.Plan(geom, data_dtype=dtype)
    plan.set_fbp_weights(w)
    pt = torch.from_numpy(p).cuda().to(plan.torch_data_dtype)
    got = plan.fbp(pt).cpu().numpy()
    want = F.fbp(geom, pt.float().cpu().numpy(), w)
    assert np.abs(want).max() > 0
    print(f"fbp {case} dtype {dtype}: rel-L2 {rel(got, want):.3e}")
    assert rel(got, want) <= TOL, rel(got, want)
    plan.close()


def _kt_errors(oat, geom, nodes, qs):
    plan = oat.Plan(geom)
    got = plan.fbp_sample_positions(nodes, qs)
    plan.close()
    want = F.sample_positions(geom, nodes, qs)
    return np.abs(got - want)


@pytest.mark.parametrize("case", sorted(CASES) + ["c2_sampled"])
def test_fbp_sample_position_accuracy(env, case):
    """The kernel's FP32 k~ (oat_fbp_sample_positions runs the arithmetic of k_fbp) against the
    FP64 definition: every (node, transducer) pair of the small cases, 400,000 sampled pairs of
    the 256^3 / 23,040-transducer scan (distances up to about 450 grid units).  The largest error
    must stay below a quarter of the guard band in which the kernel resolves k~ in double
    precision, so that outside the band its FP32 floor is the exact one."""
    torch, oat = env
    if case == "c2_sampled":
        geom = W.config("c2")
        rng = np.random.default_rng(17)
        n = 400_000
        nodes = rng.integers(0, 256, size=(n, 3))
        qs = rng.integers(0, geom.n_transducers, size=n)
    else:
        geom = CASES[case][0]()
        iz, iy, ix = np.meshgrid(np.arange(geom.nz), np.arange(geom.ny), np.arange(geom.nx), indexing="ij")
        grid = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
        nodes = np.repeat(grid, geom.n_transducers, axis=0)
        qs = np.tile(np.arange(geom.n_transducers), len(grid))
    err = _kt_errors(oat, geom, nodes, qs)
    sk = geom.spacing_mm * geom.fs_mhz / geom.c_mm_per_us
    print(f"fbp k~ error {case}: max {err.max():.3e} samples ({err.max() / sk:.3e} grid units), "
          f"rms {np.sqrt((err ** 2).mean()):.3e} samples over {len(err)} pairs; guard band {guard(geom):.3e}")
    assert np.isfinite(err).all()
    assert err.max() <= 0.25 * guard(geom), (err.max(), guard(geom))


def test_fbp_full_size_sampled_nodes(env):
    """256^3, 23,040 transducers, K = 1536: the whole volume on the GPU; 64 sampled nodes
    (through the grid and its faces) against the reference."""
    torch, oat = env
    geom = W.config("c2")
    w = F.arc_weights(geom.positions_mm, 128, 180)
    p = smooth_data(geom, seed=41, width=8.0)
    plan = oat.Plan(geom)
    plan.set_fbp_weights(w)
    got = plan.fbp(torch.from_numpy(p).cuda()).cpu().numpy()
    rng = np.random.default_rng(5)
    nodes = rng.integers(0, 256, size=(64, 3))
    nodes[:8, 0] = 0; nodes[8:16, 1] = 255; nodes[16:24, 2] = 0
    want = F.fbp(geom, p, w, nodes=nodes)
    got_s = got[nodes[:, 2], nodes[:, 1], nodes[:, 0]]
    print(f"fbp full size: rel-L2 {rel(got_s, want):.3e}")
    assert rel(got_s, want) <= TOL, rel(got_s, want)
    plan.close()


@pytest.mark.parametrize("offset", [-5e-6, -1e-6, 1e-6, 5e-6])
def test_fbp_constructed_crossing(env, offset):
    """A crossing placed on purpose: the time origin puts node 0 at k~ = n + offset samples for
    transducer 0 (inside the kernel's guard band, and for |offset| <= 5e-6 within reach of the
    FP32 error of k~), under a sharp pulse whose second difference there is large.  The kernel
    must read the pair the exact k~ selects: node 0 and the whole volume against the reference."""
    import dataclasses
    torch, oat = env
    g0 = W.make_geometry(16, 0.27, 4, 6, 7.3, 200)
    dt = 1.0 / g0.fs_mhz
    xs, ys, zs = g0.node_coords_mm()
    d = np.linalg.norm(np.array([xs[0], ys[0], zs[0]]) - g0.positions_mm[0])
    kt = (d / g0.c_mm_per_us - g0.t_min_us) / dt
    g = dataclasses.replace(g0)
    g.t_min_us = g0.t_min_us + (kt - np.floor(kt) - offset) * dt
    kt1 = F.sample_positions(g, [[0, 0, 0]], [0])[0]
    assert abs(kt1 - np.rint(kt1) - offset) < 1e-9, kt1
    t = g.t_min_us + np.arange(g.n_samples) * dt
    p = (np.exp(-0.5 * ((t[None, :] - d / g.c_mm_per_us) / (1.2 * dt)) ** 2)
         * np.linspace(0.5, 1.0, g.n_transducers)[:, None]).astype(np.float32)
    w = F.arc_weights(g.positions_mm, 4, 6)
    plan = oat.Plan(g)
    plan.set_fbp_weights(w)
    got = plan.fbp(torch.from_numpy(p).cuda()).cpu().numpy()
    plan.close()
    want = F.fbp(g, p, w)
    # the term of transducer 0 at node 0 on the other side of the integer, for scale
    wrong = dataclasses.replace(g)
    wrong.t_min_us = g.t_min_us + 2.0 * offset * dt
    alt = F.fbp(wrong, p, w)
    assert abs(alt[0, 0, 0] - want[0, 0, 0]) > 1e-3 * np.abs(want).max()       # a real crossing
    e0 = abs(got[0, 0, 0] - want[0, 0, 0]) / np.abs(want).max()
    print(f"fbp crossing at {offset:+.0e}: node 0 error {e0:.2e}, volume rel-L2 {rel(got, want):.3e}")
    assert e0 <= 1e-5 and rel(got, want) <= TOL, (e0, rel(got, want))


def test_fbp_requires_weights(env):
    torch, oat = env
    geom = W.make_geometry(8, 0.4, 2, 2, 6.0, 32)
    plan = oat.Plan(geom)
    d = torch.zeros(geom.data_shape, device="cuda")
    with pytest.raises(oat.OatError) as e:
        plan.fbp(d)
    assert e.value.code == oat.OAT_ERR_INVALID_ARG
    with pytest.raises(oat.OatError):
        plan.set_fbp_weights(np.full(geom.n_transducers, np.nan))
    with pytest.raises(ValueError):
        plan.set_fbp_weights(np.ones(3))
    plan.close()
