"""Pins of the FP64 reconstruction reference (oracle/recon.py) against closed forms and
optimality properties.  CPU only."""
import numpy as np
import pytest

from oracle import recon


def test_grad_t_is_adjoint_of_grad():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7))
    p = [rng.standard_normal((5, 6, 7)) for _ in range(3)]
    g = recon.grad(x)
    lhs = sum((g[i] * p[i]).sum() for i in range(3))
    rhs = (x * recon.grad_t(*p)).sum()
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_tv_prox_step_closed_form():
    """A volume constant in y and z with a step along x reduces isotropic TV to 1-D TV on each
    line.  1-D TV denoising (ROF) of a step a | b (a < b, m and m' points) moves the two
    plateaus by lam/m up and lam/m' down while the jump survives."""
    m, mp, a, b, lam = 5, 7, 1.0, 3.0, 0.6
    line = np.array([a] * m + [b] * mp)
    z = np.broadcast_to(line, (3, 4, m + mp)).copy()
    x = recon.tv_prox(z, lam, 3000)
    want = np.array([a + lam / m] * m + [b - lam / mp] * mp)
    assert np.allclose(x, np.broadcast_to(want, z.shape), atol=2e-4)


def test_tv_prox_special_cases():
    rng = np.random.default_rng(1)
    z = rng.standard_normal((4, 5, 6))
    assert np.array_equal(recon.tv_prox(z, 0.0, 10), np.maximum(z, 0))
    c = np.full((4, 5, 6), 0.7)
    assert np.allclose(recon.tv_prox(c, 0.3, 50), c)
    # fused gradient step: prox at z - s g
    g = rng.standard_normal(z.shape)
    assert np.allclose(recon.tv_prox(z, 0.2, 30, g=g, step=0.5), recon.tv_prox(z - 0.5 * g, 0.2, 30))


def test_tv_prox_is_a_minimiser():
    """Converged prox beats random feasible perturbations of itself on the prox objective."""
    rng = np.random.default_rng(2)
    z = np.abs(rng.standard_normal((6, 6, 6))) + 0.5 * (rng.random((6, 6, 6)) > 0.7)
    lam = 0.15
    x = recon.tv_prox(z, lam, 4000)
    f = lambda v: 0.5 * ((v - z) ** 2).sum() + lam * recon.tv(v)  # noqa: E731
    fx = f(x)
    for _ in range(50):
        d = rng.standard_normal(z.shape) * 1e-2
        assert f(np.maximum(x + d, 0.0)) >= fx - 1e-6


def test_fista_identity_operator():
    """With H = I, L = 1 and mu = 0 one FISTA step is the projection onto x >= 0."""
    rng = np.random.default_rng(3)
    u = rng.standard_normal((4, 4, 4))
    x, res = recon.fista_tv(lambda v: v, lambda v: v, u, 0.0, 1.0, 1, np.zeros_like(u))
    assert np.allclose(x, np.maximum(u, 0))
    assert res[0] == pytest.approx(np.linalg.norm(np.minimum(u, 0)) / np.linalg.norm(u))
