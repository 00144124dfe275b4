"""Pins of the resampled numerical coarse propagator G(u) = P(G_c(R u)) (oracle, the
resolution change of Sec. 4.4 applied to the numerical coarse model)."""
import numpy as np

import workloads as wl
from oracle import fd
from oracle import resample as rs


def smooth_state(M, xmax, seed):
    rng = np.random.default_rng(seed)
    X, Y = fd.mesh(M, xmax)
    a = rng.uniform(0.5, 1.5, 4)
    return a[0] * np.sin(0.7 * X + a[1]) * np.cos(0.4 * Y) + a[2] * X * Y / xmax + a[3] * Y


def test_same_grid_is_plain_coarse_propagation():
    p = wl.Params(0.3, 0.2, 0.5, 0.05, payoff=wl.BASKET)
    M, xmax = 24, 4.0
    u = smooth_state(M, xmax, 1)
    got = rs.resampled_coarse(u, xmax, p, 0.25, 0.125, 2, M)
    want = fd.ImplicitEuler(M, xmax, p, 0.0625).propagate(u, 0.25, 2)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_shared_nodes_carry_the_coarse_solution():
    # M - 1 = 2 (Mc - 1): every other fine node is a coarse node, where R samples exactly and
    # P returns the coarse value, so G(u) there is G_c(u_c); between them G(u) is the
    # bilinear interpolant.  A prolonged increment instead of a prolonged state, a transposed
    # or shifted index map all break this.
    p = wl.Params(0.25, 0.35, -0.4, 0.03, payoff=wl.EXCHANGE)
    M, Mc, xmax = 33, 17, 4.0
    u = smooth_state(M, xmax, 2)
    uc = u[::2, ::2]
    got = rs.resampled_coarse(u, xmax, p, 0.5, 0.1, 3, Mc)
    want = fd.ImplicitEuler(Mc, xmax, p, 0.1 / 3).propagate(uc, 0.5, 3)
    assert np.max(np.abs(got[::2, ::2] - want)) <= 1e-12
    mid = got[1:-1:2, 0:-1:2]          # the far edge x = xmax holds the Dirichlet data
    assert np.max(np.abs(mid - 0.5 * (got[0:-2:2, 0:-1:2] + got[2::2, 0:-1:2]))) <= 1e-12
    assert not np.allclose(got, got.T)   # the test state is not symmetric


def test_traded_asset_is_stationary():
    # V = S1 solves the Black-Scholes equation for every parameter set: with its own
    # Dirichlet data it is a fixed point of G on any coarse grid (centred differences are
    # exact on linear functions and bilinear resampling reproduces them)
    p = wl.Params(0.3, 0.25, 0.6, 0.07, payoff=wl.BASKET)
    M, Mc, xmax = 41, 13, 4.0
    X, Y = fd.mesh(M, xmax)
    got = rs.resampled_coarse(X.copy(), xmax, p, 0.0, 0.2, 2, Mc, boundary=lambda X, Y, t: X)
    assert np.max(np.abs(got - X)) <= 1e-12
