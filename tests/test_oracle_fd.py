"""Pins for the FP64 finite-difference oracle (oracle/fd.py), eq. (fd).

Each check compares the oracle with something other than itself: the continuous
PDE applied analytically to polynomials, a dense linear solve, closed-form
option prices, and a one-dimensional tridiagonal scheme.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.stats import lognorm

import workloads as wl
from oracle import closed_forms as cf
from oracle import fd

PARAM_SETS = [
    wl.Params(0.3, 0.2, 0.5, 0.05),
    wl.Params(0.25, 0.35, -0.5, 0.03),
    wl.Params(0.45, 0.15, 0.7, 0.08),
    wl.Params(0.2, 0.2, 0.0, 0.0),
]


def continuous_R_monomial(p, a, b):
    """Eq. (bse_change_variable) applied to x^a y^b, divided by x^a y^b:
    1/2 s1^2 a(a-1) + 1/2 s2^2 b(b-1) + rho s1 s2 a b + r a + r b - r."""
    return (0.5 * p.sigma1 ** 2 * a * (a - 1) + 0.5 * p.sigma2 ** 2 * b * (b - 1)
            + p.rho * p.sigma1 * p.sigma2 * a * b + p.r * (a + b - 1))


@pytest.mark.parametrize("p", PARAM_SETS)
@pytest.mark.parametrize("M,xmax", [(7, 4.0), (12, 3.0), (33, 4.0)])
def test_operator_exact_on_biquadratics(p, M, xmax):
    # Centred differences are exact on x^a y^b with a, b <= 2, and these nine
    # monomials determine all nine stencil weights at every node.
    X, Y = fd.mesh(M, xmax)
    w = fd.stencil_weights(M, xmax, p.sigma1, p.sigma2, p.rho, p.r)
    for a in range(3):
        for b in range(3):
            u = X ** a * Y ** b
            want = continuous_R_monomial(p, a, b) * u[: M - 1, : M - 1]
            got = fd.apply_R(u, w)
            scale = 1.0 + np.max(np.abs(u)) * (1.0 + p.sigma1 ** 2 + p.sigma2 ** 2) * (M - 1) ** 2
            assert np.max(np.abs(got - want)) <= 1e-13 * scale, (a, b)


@pytest.mark.parametrize("p", PARAM_SETS[:3])
@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (2, 2)])
def test_step_maps_monomial_exactly(p, a, b):
    # With Dirichlet data c(tau) x^a y^b, c(tau) = (1 - dtau kappa)^(-tau/dtau),
    # one implicit step scales x^a y^b by 1 / (1 - dtau kappa) exactly.
    M, xmax, dtau = 11, 2.0, 0.01
    kappa = continuous_R_monomial(p, a, b)
    fac = 1.0 / (1.0 - dtau * kappa)

    def g(X, Y, tau):
        return fac ** (tau / dtau) * X ** a * Y ** b

    ie = fd.ImplicitEuler(M, xmax, p, dtau, boundary=g)
    X, Y = fd.mesh(M, xmax)
    u0 = X ** a * Y ** b
    u1 = ie.step(u0, dtau)
    u3 = ie.propagate(u0, 0.0, 3)
    assert np.max(np.abs(u1 - fac * u0)) <= 1e-12 * (1 + np.max(np.abs(u0)))
    assert np.max(np.abs(u3 - fac ** 3 * u0)) <= 1e-11 * (1 + np.max(np.abs(u0)))


@pytest.mark.parametrize("M", [4, 5, 7])
@pytest.mark.parametrize("p", PARAM_SETS[:3])
def test_step_against_dense_solve(M, p):
    # Dense brute force: build I - dtau R_h column by column from apply_R on unit
    # vectors (apply_R is pinned above), move Dirichlet data to the right-hand side
    # the same way, and solve with numpy.linalg.solve.
    xmax, dtau = 4.0, 0.05
    p = wl.Params(p.sigma1, p.sigma2, p.rho, p.r, payoff=wl.BASKET)
    ie = fd.ImplicitEuler(M, xmax, p, dtau)
    w = fd.stencil_weights(M, xmax, p.sigma1, p.sigma2, p.rho, p.r)
    n = M - 1
    A = np.zeros((n * n, n * n))
    for k in range(n * n):
        e = np.zeros((M, M))
        e[k // n, k % n] = 1.0
        A[:, k] = e[:n, :n].ravel() - dtau * fd.apply_R(e, w).ravel()
    rng = np.random.default_rng(M)
    u0 = rng.uniform(0.0, 2.0, (M, M))
    gb = ie.boundary_values(dtau)
    bd = gb.copy()
    bd[:n, :n] = 0.0
    rhs = u0[:n, :n].ravel() + dtau * fd.apply_R(bd, w).ravel()
    want = np.linalg.solve(A, rhs).reshape(n, n)
    got = ie.step(u0, dtau)
    assert np.max(np.abs(got[:n, :n] - want)) <= 1e-12
    assert np.array_equal(got[n, :], gb[n, :]) and np.array_equal(got[:, n], gb[:, n])


def thomas_bs1d(M, xmax, sigma, r, K, dtau, nsteps):
    """1-D Black-Scholes call by implicit Euler with centred differences, solved
    with the tridiagonal (Thomas) algorithm; Dirichlet at x = xmax from the closed
    form; at x = 0 the PDE row reduces to u_tau = -r u."""
    x = np.arange(M) * (xmax / (M - 1))
    h = x[1] - x[0]
    u = np.maximum(x - K, 0.0)
    out = [u.copy()]
    lo = -dtau * (0.5 * sigma ** 2 * x ** 2 / h ** 2 - r * x / (2 * h))
    di = 1.0 + dtau * (sigma ** 2 * x ** 2 / h ** 2 + r)
    up = -dtau * (0.5 * sigma ** 2 * x ** 2 / h ** 2 + r * x / (2 * h))
    for m in range(nsteps):
        tau = (m + 1) * dtau
        gR = float(cf.bs_call_1d(np.array([xmax]), K, r, sigma, tau)[0])
        n = M - 1
        a, bb, c, d = lo[:n].copy(), di[:n].copy(), up[:n].copy(), u[:n].copy()
        d[n - 1] -= c[n - 1] * gR
        for i in range(1, n):
            f = a[i] / bb[i - 1]
            bb[i] -= f * c[i - 1]
            d[i] -= f * d[i - 1]
        sol = np.zeros(n)
        sol[n - 1] = d[n - 1] / bb[n - 1]
        for i in range(n - 2, -1, -1):
            sol[i] = (d[i] - c[i] * sol[i + 1]) / bb[i]
        u = np.concatenate([sol, [gR]])
        out.append(u.copy())
    return x, np.array(out)


def test_one_asset_reduction():
    # A payoff in x only with y-independent Dirichlet data gives a y-independent
    # solution equal to the 1-D scheme; the 1-D scheme tracks the closed form.
    M, xmax, sigma, r, K = 41, 4.0, 0.3, 0.05, 1.0
    nsteps, dtau = 40, 1.0 / 40
    x, hist = thomas_bs1d(M, xmax, sigma, r, K, dtau, nsteps)
    table = {round(k * dtau, 12): hist[k] for k in range(nsteps + 1)}

    def g(X, Y, tau):
        return np.broadcast_to(table[round(tau, 12)][None, :], X.shape).copy()

    p = wl.Params(sigma, 0.37, 0.6, r, 1.0, K, payoff=wl.CALL1)
    ie = fd.ImplicitEuler(M, xmax, p, dtau, boundary=g)
    X, Y = fd.mesh(M, xmax)
    u = fd.payoff(p, X, Y)
    u = ie.propagate(u, 0.0, nsteps)
    assert np.max(np.abs(u - hist[-1][None, :])) <= 1e-12
    exact = cf.bs_call_1d(x, K, r, sigma, 1.0)
    inner = (x > 0.5) & (x < 2.5)
    assert np.max(np.abs(hist[-1][inner] - exact[inner])) < 5e-3


def test_margrabe_convergence():
    # Exchange option with Margrabe Dirichlet data: the error against the closed
    # form on [1, 3]^2 falls like O(h^2 + dtau) when h halves and dtau quarters.
    T = 0.5
    p = wl.Params(0.25, 0.35, 0.3, 0.03, T, payoff=wl.EXCHANGE)
    errs = []
    for M, steps in [(17, 8), (33, 32), (65, 128)]:
        ie = fd.ImplicitEuler(M, 4.0, p, T / steps)
        X, Y = fd.mesh(M, 4.0)
        u = ie.propagate(fd.payoff(p, X, Y), 0.0, steps)
        ex = cf.margrabe(X, Y, p.sigma1, p.sigma2, p.rho, T)
        box = (X >= 1.0) & (X <= 3.0) & (Y >= 1.0) & (Y <= 3.0)
        errs.append(np.max(np.abs(u - ex)[box]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


def test_gershgorin_contraction_matches_dense():
    p = PARAM_SETS[0]
    M, xmax, dtau = 6, 4.0, 0.02
    w = fd.stencil_weights(M, xmax, p.sigma1, p.sigma2, p.rho, p.r)
    n = M - 1
    A = np.zeros((n * n, n * n + 2 * M))
    # dense rows of I - dtau R_h including couplings to Dirichlet nodes
    full = np.zeros((n * n, M * M))
    for k in range(M * M):
        e = np.zeros((M, M))
        e.flat[k] = 1.0
        col = -dtau * fd.apply_R(e, w).ravel()
        full[:, k] = col
    for r_ in range(n * n):
        j, i = divmod(r_, n)
        full[r_, j * M + i] += 1.0
    diag = np.array([full[r_, (r_ // n) * M + r_ % n] for r_ in range(n * n)])
    off = np.abs(full).sum(axis=1) - np.abs(diag)
    assert math.isclose(np.max(off / np.abs(diag)), fd.jacobi_contraction(M, xmax, p, dtau), rel_tol=1e-12)


def test_initial_payoffs():
    X, Y = fd.mesh(5, 4.0)
    pb = wl.Params(0.3, 0.2, 0.5, 0.05, strike=1.0, payoff=wl.BASKET)
    assert np.array_equal(fd.payoff(pb, X, Y), np.maximum(0.5 * X + 0.5 * Y - 1.0, 0.0))
    pe = wl.Params(0.3, 0.2, 0.5, 0.05, payoff=wl.EXCHANGE)
    assert fd.payoff(pe, X, Y)[0, 4] == 4.0 and fd.payoff(pe, X, Y)[4, 0] == 0.0
