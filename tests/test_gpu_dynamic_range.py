"""Backprojector precision at adversarial dynamic range (the fixed-point units of H^T).

H^T (the adjoint of Eqs. dis_srt and dis_g2p) accumulates exact fixed-point integers whose units
come from the data: per pass of transducers, from that pass's largest |D^T y|, and a pass ends
early before a transducer whose largest |D^T y| is more than 2^8 away from the pass's.  These
cases hold it to the 1e-5 relative L2 bar against the FP64 oracle where one unit for the whole
call, set by the largest value, would lose bits:
  - t_min = 0 with K = 1536 samples: the D^T weights C_D / tau_k span three orders of magnitude
    over the record, and the early samples' shells never reach the grid;
  - one sample 1e4 and 1e6 times the rest, alone in its transducer row: besides the relative L2
    over the volume, the error on the nodes that the spike's shells do not touch (where the
    oracle's response to the spike is exactly zero) is held to 1e-5 of the response there -- a
    unit set by the spike would miss that by about 30x at 1e6;
  - the same spike inside a noisy row: the relative L2 over the volume (the row's other samples
    share the spike's pass and keep about 10 bits of it, which is printed);
  - a late reconstruction residual: the response to a small structured correction plus white
    noise three orders of magnitude below it."""
import numpy as np
import pytest

import oracle
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


def backproject(env, geom, y):
    torch, oat = env
    plan = oat.Plan(geom)
    a = plan.backproject(torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()).cpu().numpy()
    plan.close()
    return a.astype(np.float64)


def test_tmin0_long_record(env):
    """64^3 @ 0.2 mm, 8 x 8 transducers on 20 mm, K = 1536 from t = 0: H, H^T and the adjoint
    identity against the oracle."""
    torch, oat = env
    geom = W.make_geometry(64, 0.2, 8, 8, 20.0, 1536, t_min_us=0.0)
    alpha = W.spheres_phantom(geom, 6, seed=41)
    y = W.random_data(geom, seed=42)
    plan = oat.Plan(geom)
    u = plan.project(torch.from_numpy(alpha).cuda()).cpu().numpy().astype(np.float64)
    a = plan.backproject(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    plan.close()
    eu, ea = rel(u, oracle.H(geom, alpha)), rel(a, oracle.Ht(geom, y))
    adj = abs(float((u * y).sum()) - float((alpha.astype(np.float64) * a).sum())) / (np.linalg.norm(u) * np.linalg.norm(y))
    print(f"t_min = 0, K = 1536: H {eu:.3e}, H^T {ea:.3e}, adjoint {adj:.3e}")
    assert eu <= TOL and ea <= TOL and adj <= TOL, (eu, ea, adj)


SPIKE_GEOM = dict(n=32, spacing_mm=0.25, rings=4, views=8, radius_mm=9.0, n_samples=160)


def _spike_data(geom, amp, in_noisy_row, q_s=5):
    y = W.random_data(geom, seed=51).astype(np.float64)
    k_s = geom.n_samples // 2                  # the window is centred on the arrival from the centre
    spike = np.zeros_like(y)
    spike[q_s, k_s] = amp
    if not in_noisy_row:
        y[q_s] = 0.0
    return (y + spike).astype(np.float32), spike


@pytest.mark.parametrize("amp", [1e4, 1e6])
def test_isolated_spike_costs_the_rest_nothing(env, amp):
    geom = W.make_geometry(SPIKE_GEOM["n"], SPIKE_GEOM["spacing_mm"], SPIKE_GEOM["rings"], SPIKE_GEOM["views"],
                           SPIKE_GEOM["radius_mm"], SPIKE_GEOM["n_samples"])
    y, spike = _spike_data(geom, amp, in_noisy_row=False)
    got = backproject(env, geom, y)
    want = oracle.Ht(geom, y)
    far = oracle.Ht(geom, spike) == 0.0       # nodes no lattice point of the spike's shells touches
    assert far.sum() > 0.5 * far.size and (~far).sum() > 0
    e_all, e_far = rel(got, want), rel(got[far], want[far])
    print(f"isolated spike {amp:.0e}: rel-L2 {e_all:.3e}, away from the spike's shells {e_far:.3e}")
    assert e_all <= TOL and e_far <= TOL, (e_all, e_far)


@pytest.mark.parametrize("amp", [1e4, 1e6])
def test_spike_in_noisy_row(env, amp):
    geom = W.make_geometry(SPIKE_GEOM["n"], SPIKE_GEOM["spacing_mm"], SPIKE_GEOM["rings"], SPIKE_GEOM["views"],
                           SPIKE_GEOM["radius_mm"], SPIKE_GEOM["n_samples"])
    y, spike = _spike_data(geom, amp, in_noisy_row=True)
    got = backproject(env, geom, y)
    want = oracle.Ht(geom, y)
    far = oracle.Ht(geom, spike) == 0.0
    e_all, e_far = rel(got, want), rel(got[far], want[far])
    print(f"spike {amp:.0e} in a noisy row: rel-L2 {e_all:.3e} (away from the spike's shells {e_far:.3e})")
    assert e_all <= TOL, e_all


def test_late_residual(env):
    """y = 1e-4 H(delta) + 1e-7 N(0, 1): the response to a small smooth correction delta (the
    structure a late FISTA residual keeps) plus white noise a thousand times smaller."""
    geom = W.config("small")
    rng = np.random.default_rng(61)
    delta = W.random_volume(geom, seed=62).astype(np.float64)
    for ax in range(3):                                     # smooth it: three box filters per axis
        for _ in range(3):
            delta = (np.roll(delta, 1, ax) + delta + np.roll(delta, -1, ax)) / 3.0
    y = (1e-4 * oracle.H(geom, delta) + 1e-7 * rng.standard_normal(geom.data_shape)).astype(np.float32)
    got = backproject(env, geom, y)
    e = rel(got, oracle.Ht(geom, y))
    print(f"late residual: rel-L2 {e:.3e}")
    assert e <= TOL, e
