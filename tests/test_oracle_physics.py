"""Pins of the physics-informed loss oracle (Sec. 3.5, eq. bs_totalloss: the PDE term)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fd, physics


def _params(sigma1=0.3, sigma2=0.2, rho=0.5, r=0.05, payoff=wl.BASKET):
    return wl.Params(sigma1, sigma2, rho, r, payoff=payoff)


@pytest.mark.parametrize("M,rho", [(9, 0.5), (17, -0.6)])
def test_exact_implicit_step_has_zero_residual(M, rho):
    # the slice predicted by one exact implicit-Euler step of eq. (fd) satisfies the
    # discretised PDE at every collocation point
    p = _params(rho=rho)
    dtau = 0.05
    u0 = fd.initial_state(M, 4.0, p)
    u1 = fd.ImplicitEuler(M, 4.0, p, dtau).step(u0, dtau)
    w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
    r = physics.residual(u1, u0, dtau, w)
    assert np.max(np.abs(r)) <= 1e-9 * np.max(np.abs(u1)) / dtau
    assert physics.loss(u1, u0, dtau, w) <= 1e-18 * np.max(np.abs(u1)) ** 2 / dtau ** 2


def test_residual_of_a_biquadratic_is_the_closed_form():
    # u = x^2 y: centred differences are exact, and R u = (s1^2 + 2 rho s1 s2 + 2 r) x^2 y in
    # closed form; with u_prev = u - dtau (R u + c) the residual is c at every collocation point
    M, xmax, dtau, c = 11, 4.0, 0.1, 0.37
    p = _params(sigma1=0.4, sigma2=0.25, rho=0.3, r=0.07)
    X, Y = fd.mesh(M, xmax)
    u = X ** 2 * Y
    Ru = (p.sigma1 ** 2 + 2 * p.rho * p.sigma1 * p.sigma2 + 2 * p.r) * X ** 2 * Y
    u_prev = u - dtau * (Ru + c)
    w = fd.stencil_weights(M, xmax, p.sigma1, p.sigma2, p.rho, p.r)
    r = physics.residual(u, u_prev, dtau, w)
    assert r.shape == (M - 1, M - 1)
    np.testing.assert_allclose(r, c, rtol=0, atol=1e-11)
    assert abs(physics.loss(u, u_prev, dtau, w) - c * c) <= 1e-11


@pytest.mark.parametrize("M", [5, 7])
def test_gradient_matches_finite_differences(M):
    # brute force: central differences of the loss at every node of a tiny grid
    rng = np.random.default_rng(3)
    p = _params(rho=-0.4)
    dtau = 0.02
    w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
    u_pred = rng.standard_normal((M, M))
    u_prev = rng.standard_normal((M, M))
    g = physics.loss_grad(u_pred, u_prev, dtau, w)
    eps = 1e-6
    fdg = np.zeros((M, M))
    for j in range(M):
        for i in range(M):
            up = u_pred.copy(); up[j, i] += eps
            um = u_pred.copy(); um[j, i] -= eps
            fdg[j, i] = (physics.loss(up, u_prev, dtau, w) - physics.loss(um, u_prev, dtau, w)) / (2 * eps)
    np.testing.assert_allclose(g, fdg, rtol=1e-6, atol=1e-6 * np.max(np.abs(fdg)))
    # the far edges hold no collocation point but are read by their neighbours' rows
    assert np.all(g[M - 1, :] != 0.0) and np.all(g[:, M - 1] != 0.0)


def _fd_gradient(loss_fn, u_pred, eps=1e-6):
    M = u_pred.shape[0]
    out = np.zeros((M, M))
    for j in range(M):
        for i in range(M):
            up = u_pred.copy(); up[j, i] += eps
            um = u_pred.copy(); um[j, i] -= eps
            out[j, i] = (loss_fn(up) - loss_fn(um)) / (2 * eps)
    return out


@pytest.mark.parametrize("kind", ["offset_sign", "missing_diag", "no_dtau"])
def test_planted_gradient_mistakes_fail_the_finite_difference_pin(kind):
    # plausible slips in writing the adjoint (the scatter to the negated offset, the
    # dropped 1/dtau identity part, a factor dtau too many) must disagree with the
    # finite differences that pin the correct gradient
    M, dtau = 6, 0.02
    rng = np.random.default_rng(4)
    p = _params(rho=0.6)
    w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
    u_pred = rng.standard_normal((M, M))
    u_prev = rng.standard_normal((M, M))
    n = M - 1
    r = physics.residual(u_pred, u_prev, dtau, w)
    c = 2.0 * r / (n * n)
    g = np.zeros((M, M))
    if kind != "missing_diag":
        g[:n, :n] += c / dtau * (dtau if kind == "no_dtau" else 1.0)
    J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for (di, dj), wt in w.items():
        sgn = -1 if kind == "offset_sign" else 1
        tj, ti = J + sgn * dj, I + sgn * di
        ok = (tj >= 0) & (ti >= 0) & (tj < M) & (ti < M)
        np.add.at(g, (tj[ok], ti[ok]), -(c * wt[:n, :n])[ok])
    want = _fd_gradient(lambda u: physics.loss(u, u_prev, dtau, w), u_pred)
    assert np.max(np.abs(g - want)) > 1e-3 * np.max(np.abs(want))
    np.testing.assert_allclose(physics.loss_grad(u_pred, u_prev, dtau, w), want, rtol=1e-6,
                               atol=1e-6 * np.max(np.abs(want)))
