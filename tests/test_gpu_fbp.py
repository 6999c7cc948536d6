"""Parity of the sm_103a filtered backprojection (oat_fbp, through the C ABI) with the FP64
reference oracle/fbp.py (Eq. disfbp).

Tolerance 1e-5 relative L2: per term the kernel keeps the sample position to about 1e-6 of a
sample (float-pair distance to each brick centre, small FP32 offsets) and sums with
compensation, so its error stays near FP32 rounding of the data and weights.  FP16 / BF16 data
are read exactly, so the reference gets the same rounded values.

Eq. disfbp is discontinuous in the sample position: where k~ crosses an integer the one-sided
difference p_{k+1} - p_k moves to the next pair, so a rounding difference that moves k~ across
an integer changes that term by the second difference of the data.  The kernel's k~ error is
measured directly (oat_fbp_sample_positions against the FP64 definition, `kt_max`); where the
exact k~ lies within twice that error bound of a sample both sides are readings the FP32 kernel may
take, so the comparison allows each node the reference's total change over such pairs
(`ambiguity`) and holds everything else to the tolerance.  The raw error is printed beside it.
The data are band-limited, as measured pressure is (Gaussian pulses several samples wide, or the
forward model's data of an object): for white noise the second difference is as large as the
data."""
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


def rel_beyond(got, want, amb):
    """Relative L2 of the part of got - want that the integer-crossing allowance amb does not
    explain."""
    d = np.maximum(np.abs(np.asarray(got, np.float64) - want) - amb, 0.0)
    return float(np.linalg.norm(d) / np.linalg.norm(want))


# The kernel's k~ error is a distance error: measured by test_fbp_sample_position_accuracy on
# every small case and on sampled pairs of the 256^3 / 23,040-transducer scan at 1.1e-6 to 1.9e-6
# grid units at most (rms 2.5e-7), bounded here by KT_GRID grid units, i.e. KT_GRID ds / (c dt)
# samples.  The window of the integer-crossing allowance is twice that bound.
KT_GRID = 2.2e-6


def kt_max(geom):
    """Bound of the kernel's k~ error in samples for this geometry."""
    return KT_GRID * geom.spacing_mm * geom.fs_mhz / geom.c_mm_per_us


def eps_k(geom):
    return 2.0 * kt_max(geom)


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
    n_r = {"ragged": 3, "tmin0": 2, "window_cut": 3, "physical": 6, "physical_spheres": 6, "coarse_direct": 3}[case]
    n_v = geom.n_transducers // n_r
    w = F.arc_weights(geom.positions_mm, n_r, n_v)
    p = _data(geom, kind, 11)
    plan = oat.Plan(geom, data_dtype=dtype)
    plan.set_fbp_weights(w)
    pt = torch.from_numpy(p).cuda().to(plan.torch_data_dtype)
    got = plan.fbp(pt).cpu().numpy()
    want, amb = F.fbp(geom, pt.float().cpu().numpy(), w, ambiguity=eps_k(geom))
    assert np.abs(want).max() > 0
    print(f"fbp {case} dtype {dtype}: raw rel-L2 {rel(got, want):.3e}, beyond the allowance "
          f"{rel_beyond(got, want, amb):.3e}")
    assert rel_beyond(got, want, amb) <= TOL, (rel(got, want), rel_beyond(got, want, amb))
    plan.close()


def _kt_errors(oat, geom, nodes, qs):
    plan = oat.Plan(geom)
    got = plan.fbp_sample_positions(nodes, qs)
    plan.close()
    want = F.sample_positions(geom, nodes, qs)
    return np.abs(got - want)


@pytest.mark.parametrize("case", sorted(CASES) + ["c2_sampled"])
def test_fbp_sample_position_accuracy(env, case):
    """The kernel's own k~ (oat_fbp_sample_positions runs the arithmetic of k_fbp) against the
    FP64 definition: every (node, transducer) pair of the small cases, 400,000 sampled pairs of
    the 256^3 / 23,040-transducer scan (distances up to about 450 grid units).  The largest error
    bounds the integer-crossing window used by the parity tests (twice the bound)."""
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
          f"rms {np.sqrt((err ** 2).mean()):.3e} samples over {len(err)} pairs; bound {kt_max(geom):.3e}")
    assert np.isfinite(err).all()
    assert err.max() <= kt_max(geom), (err.max(), kt_max(geom))


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
    want, amb = F.fbp(geom, p, w, nodes=nodes, ambiguity=eps_k(geom))
    got_s = got[nodes[:, 2], nodes[:, 1], nodes[:, 0]]
    print(f"fbp full size: raw rel-L2 {rel(got_s, want):.3e}, beyond the allowance {rel_beyond(got_s, want, amb):.3e}")
    assert rel_beyond(got_s, want, amb) <= TOL, (rel(got_s, want), rel_beyond(got_s, want, amb))
    plan.close()


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
