"""Pins for oracle/closed_forms.py against independent mathematics."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.stats import multivariate_normal, norm

from oracle import closed_forms as cf


def test_bs_call_matches_lognormal_expectation():
    # V = e^{-r tau} E[max(S_tau - K, 0)], S_tau lognormal with drift r.
    x, K, r, s, tau = 1.3, 1.0, 0.05, 0.3, 0.8
    mu = math.log(x) + (r - 0.5 * s * s) * tau
    sd = s * math.sqrt(tau)
    f = lambda z: max(math.exp(mu + sd * z) - K, 0.0) * norm.pdf(z)
    want = math.exp(-r * tau) * quad(f, -12, 12, points=[(math.log(K) - mu) / sd], limit=200)[0]
    got = float(cf.bs_call_1d(np.array([x]), K, r, s, tau)[0])
    assert abs(got - want) < 1e-9


def test_bs_call_limits():
    x = np.array([0.0, 0.5, 2.0])
    assert np.array_equal(cf.bs_call_1d(x, 1.0, 0.05, 0.3, 0.0), np.maximum(x - 1.0, 0.0))
    assert cf.bs_call_1d(np.array([0.0]), 1.0, 0.05, 0.3, 1.0)[0] == 0.0


def test_margrabe_symmetry_and_pde():
    s1, s2, rho, tau = 0.25, 0.35, -0.5, 0.7
    x, y = 1.7, 1.2
    # exchange parity: V(x, y) - V(y, x) = x - y  (with the roles of the assets swapped)
    v_xy = float(cf.margrabe(x, y, s1, s2, rho, tau))
    v_yx = float(cf.margrabe(y, x, s2, s1, rho, tau))
    assert abs((v_xy - v_yx) - (x - y)) < 1e-13
    # the closed form satisfies eq. (bse_change_variable) (central differences, FP64)
    r = 0.04
    h, dt = 1e-3, 1e-5
    V = lambda a, b, t: float(cf.margrabe(a, b, s1, s2, rho, t))
    u_t = (V(x, y, tau + dt) - V(x, y, tau - dt)) / (2 * dt)
    u_xx = (V(x + h, y, tau) - 2 * V(x, y, tau) + V(x - h, y, tau)) / h ** 2
    u_yy = (V(x, y + h, tau) - 2 * V(x, y, tau) + V(x, y - h, tau)) / h ** 2
    u_xy = (V(x + h, y + h, tau) - V(x + h, y - h, tau) - V(x - h, y + h, tau) + V(x - h, y - h, tau)) / (4 * h * h)
    u_x = (V(x + h, y, tau) - V(x - h, y, tau)) / (2 * h)
    u_y = (V(x, y + h, tau) - V(x, y - h, tau)) / (2 * h)
    res = (u_t - 0.5 * s1 ** 2 * x * x * u_xx - 0.5 * s2 ** 2 * y * y * u_yy
           - rho * s1 * s2 * x * y * u_xy - r * x * u_x - r * y * u_y + r * V(x, y, tau))
    assert abs(res) < 1e-5


def test_margrabe_edges():
    assert float(cf.margrabe(2.0, 0.0, 0.3, 0.2, 0.5, 1.0)) == 2.0
    assert float(cf.margrabe(0.0, 2.0, 0.3, 0.2, 0.5, 1.0)) == 0.0
    assert float(cf.margrabe(3.0, 1.0, 0.3, 0.2, 0.5, 0.0)) == 2.0


@pytest.mark.parametrize("rho", [-0.7, -0.2, 0.3, 0.5, 0.85])
def test_bvn_against_scipy(rho):
    pts = [(-1.0, 0.5), (0.3, 0.3), (1.5, -0.4), (2.0, 2.5), (-2.5, -1.0)]
    for h, k in pts:
        want = multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]]).cdf([h, k])
        got = float(cf.bvn_cdf(h, k, rho))
        assert abs(got - want) < 2e-6, (h, k)


@pytest.mark.parametrize("rho", [-0.6, 0.0, 0.5, 0.9])
def test_bvn_sheppard(rho):
    # B(0, 0; rho) = 1/4 + arcsin(rho) / (2 pi)  (Sheppard's formula)
    assert abs(float(cf.bvn_cdf(0.0, 0.0, rho)) - (0.25 + math.asin(rho) / (2 * math.pi))) < 1e-13


def test_cash_or_nothing_limits():
    # rho = 0 factorises into two one-asset digitals; tau = 0 gives the payoff.
    S1 = S2 = 100.0
    x, y, r, s1, s2, tau = 110.0, 95.0, 0.05, 0.3, 0.25, 0.5
    d1 = (math.log(x / S1) + (r - 0.5 * s1 ** 2) * tau) / (s1 * math.sqrt(tau))
    d2 = (math.log(y / S2) + (r - 0.5 * s2 ** 2) * tau) / (s2 * math.sqrt(tau))
    want = math.exp(-r * tau) * norm.cdf(d1) * norm.cdf(d2)
    assert abs(float(cf.cash_or_nothing(x, y, S1, S2, 1.0, r, s1, s2, 0.0, tau)) - want) < 1e-14
    pay = cf.cash_or_nothing(np.array([99.0, 100.0, 120.0]), np.array([120.0, 100.0, 99.0]),
                             S1, S2, 2.0, r, s1, s2, 0.5, 0.0)
    assert np.array_equal(pay, [0.0, 2.0, 0.0])
