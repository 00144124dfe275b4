"""Pins of the n-asset oracle (eq. bse_general discretised like eq. fd), CPU only.

- n = 2 reproduces the two-asset oracle (separately written): stencil weights and a step;
- n = 3: the discrete operator equals the continuous one on all 27 monomials x^a y^b z^c
  (a, b, c <= 2), which fixes every weight of the 19-point stencil, each cross pair's sign
  and scale included; a planted sign error in one pair is caught;
- discrete eigenfunctions: one implicit step multiplies 1, x_2, x_3^2 and x_1 x_2 x_3 by
  1 / (1 - dtau kappa) exactly;
- a payoff that does not depend on asset 3 gives, plane by plane, the two-asset solution:
  every difference along asset 3 vanishes, whatever sigma_3 and rho_13, rho_23;
- on a tiny grid the sparse system equals the dense operator built column by column.
"""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import fd
from oracle import fd_nd

SIG3 = [0.3, 0.2, 0.25]
RHO3 = np.array([[1.0, 0.5, -0.3], [0.5, 1.0, 0.2], [-0.3, 0.2, 1.0]])
R = 0.05
XMAX = 4.0


def test_two_assets_is_the_two_asset_scheme():
    M = 17
    p = wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE)
    w2 = fd.stencil_weights(M, XMAX, p.sigma1, p.sigma2, p.rho, p.r)
    wn = fd_nd.stencil_weights(M, XMAX, [p.sigma1, p.sigma2], [[1.0, p.rho], [p.rho, 1.0]], p.r)
    # axis offsets (y, x) of the n-asset arrays are (dj, di) of the two-asset ones
    assert {(o[1], o[0]) for o in wn} == set(w2)
    for (dy, dx), wt in wn.items():
        np.testing.assert_allclose(wt, w2[(dx, dy)], rtol=1e-15, atol=1e-12)
    dtau = 0.01
    ie2 = fd.ImplicitEuler(M, XMAX, p, dtau)
    g2 = fd.dirichlet(p)
    ien = fd_nd.ImplicitEulerND(M, XMAX, [p.sigma1, p.sigma2], [[1.0, p.rho], [p.rho, 1.0]], p.r, dtau,
                                lambda X, tau: g2(X[0], X[1], tau))
    u0 = fd.initial_state(M, XMAX, p)
    np.testing.assert_allclose(ien.step(u0, 0.3), ie2.step(u0, 0.3), rtol=0, atol=1e-13)


def continuous_R(a, b, c, X, sig, rho, r):
    """The continuous operator of eq. bse_general on x^a y^b z^c, by hand."""
    e = (a, b, c)
    xs = X

    def mono(exps):
        out = np.ones_like(xs[0])
        for x, k in zip(xs, exps):
            out = out * (x ** k if k > 0 else 1.0)
        return out

    u = mono(e)
    out = -r * u
    for p in range(3):
        if e[p] >= 1:
            d = list(e); d[p] -= 1
            out = out + r * xs[p] * e[p] * mono(d)
        if e[p] >= 2:
            d = list(e); d[p] -= 2
            out = out + 0.5 * sig[p] ** 2 * xs[p] ** 2 * e[p] * (e[p] - 1) * mono(d)
    for p, q in itertools.combinations(range(3), 2):
        if e[p] >= 1 and e[q] >= 1:
            d = list(e); d[p] -= 1; d[q] -= 1
            out = out + rho[p][q] * sig[p] * sig[q] * xs[p] * xs[q] * e[p] * e[q] * mono(d)
    return out


def monomial(a, b, c, X):
    return X[0] ** a * X[1] ** b * X[2] ** c


@pytest.mark.parametrize("M", [6, 9])
def test_quadratic_monomials_exact(M):
    X = fd_nd.coords(M, XMAX, 3)
    w = fd_nd.stencil_weights(M, XMAX, SIG3, RHO3, R)
    core = (slice(0, M - 1),) * 3
    for a, b, c in itertools.product(range(3), repeat=3):
        got = fd_nd.apply_R(monomial(a, b, c, X), w)
        want = continuous_R(a, b, c, X, SIG3, RHO3, R)[core]
        assert np.max(np.abs(got - want)) <= 1e-11 * max(1.0, np.max(np.abs(want))), (a, b, c)


def test_planted_cross_sign_error_is_caught():
    M = 7
    X = fd_nd.coords(M, XMAX, 3)
    w = fd_nd.stencil_weights(M, XMAX, SIG3, RHO3, R)
    bad = {k: np.array(v, copy=True) for k, v in w.items()}
    # flip the (x_1, x_3) cross pair: offsets along axes 2 (asset 1) and 0 (asset 3)
    for off in [(1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1)]:
        bad[off] = -bad[off]
    core = (slice(0, M - 1),) * 3
    got = fd_nd.apply_R(monomial(1, 0, 1, X), bad)
    want = continuous_R(1, 0, 1, X, SIG3, RHO3, R)[core]
    assert np.max(np.abs(got - want)) > 1e-3


@pytest.mark.parametrize("exps,kappa", [
    ((0, 0, 0), -R),
    ((0, 1, 0), 0.0),
    ((0, 0, 2), SIG3[2] ** 2 + R),
    ((1, 1, 1), RHO3[0][1] * SIG3[0] * SIG3[1] + RHO3[0][2] * SIG3[0] * SIG3[2]
     + RHO3[1][2] * SIG3[1] * SIG3[2] + 2 * R),
])
def test_eigen_monomials_one_step(exps, kappa):
    M, dtau = 8, 0.02
    lam = 1.0 / (1.0 - dtau * kappa)
    X = fd_nd.coords(M, XMAX, 3)
    u = monomial(*exps, X)
    ie = fd_nd.ImplicitEulerND(M, XMAX, SIG3, RHO3, R, dtau,
                               lambda Xs, tau: lam * monomial(*exps, Xs))
    got = ie.step(u, dtau)
    assert np.max(np.abs(got - lam * u)) <= 1e-12 * max(1.0, np.max(np.abs(u)))


def test_payoff_without_asset3_reduces_to_two_assets():
    M, dtau, steps = 11, 0.01, 5
    p = wl.Params(SIG3[0], SIG3[1], RHO3[0][1], R, payoff=wl.EXCHANGE)
    ie2 = fd.ImplicitEuler(M, XMAX, p, dtau)
    u2 = fd.initial_state(M, XMAX, p)
    holder = {}
    ie3 = fd_nd.ImplicitEulerND(M, XMAX, SIG3, RHO3, R, dtau,
                                lambda Xs, tau: np.broadcast_to(holder["u2"], Xs[0].shape))
    u3 = np.broadcast_to(u2, (M, M, M)).copy()
    for s in range(steps):
        tau = (s + 1) * dtau
        u2 = ie2.step(u2, tau)
        holder["u2"] = u2          # the far faces, asset 3's included, carry the 2-D solution
        u3 = ie3.step(u3, tau)
        assert np.max(np.abs(u3 - u2[None, :, :])) <= 1e-12 * np.max(np.abs(u2))


def test_tiny_grid_sparse_equals_dense():
    M, dtau = 4, 0.05
    m = M - 1
    w = fd_nd.stencil_weights(M, XMAX, SIG3, RHO3, R)
    # dense I - dtau R_h on the PDE nodes, column by column from apply_R (far faces zero)
    A = np.zeros((m ** 3, m ** 3))
    for col in range(m ** 3):
        e = np.zeros((M, M, M))
        e[np.unravel_index(col, (m, m, m))] = 1.0
        A[:, col] = e[:m, :m, :m].ravel() - dtau * fd_nd.apply_R(e, w).ravel()
    ie = fd_nd.ImplicitEulerND(M, XMAX, SIG3, RHO3, R, dtau, lambda Xs, tau: np.zeros_like(Xs[0]))
    np.testing.assert_allclose(ie.A.toarray(), A, rtol=0, atol=1e-13)
    rng = np.random.default_rng(5)
    u = np.zeros((M, M, M))
    u[:m, :m, :m] = rng.standard_normal((m, m, m))
    got = ie.step(u, dtau)
    want = np.linalg.solve(A, u[:m, :m, :m].ravel())
    np.testing.assert_allclose(got[:m, :m, :m].ravel(), want, rtol=0, atol=1e-12)
