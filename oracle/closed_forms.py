"""Closed-form option prices used as far-field Dirichlet data and as checks.

Test infrastructure only (see ``oracle/__init__``).  FP64 throughout.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr


def bs_call_1d(x, K, r, sigma, tau):
    """European call on one asset, V = x N(d1) - K e^{-r tau} N(d2).

    The one-asset special case of eq. (bse) (Black and Scholes 1973).  At tau = 0
    it is the payoff max(x - K, 0); at x = 0 it is 0.
    """
    x = np.asarray(x, dtype=np.float64)
    if tau <= 0.0:
        return np.maximum(x - K, 0.0)
    out = np.zeros_like(x)
    pos = x > 0.0
    sq = sigma * math.sqrt(tau)
    xp = x[pos]
    d1 = (np.log(xp / K) + (r + 0.5 * sigma * sigma) * tau) / sq
    d2 = d1 - sq
    out[pos] = xp * ndtr(d1) - K * math.exp(-r * tau) * ndtr(d2)
    return out


def margrabe(x, y, sigma1, sigma2, rho, tau):
    """Exchange option max(x - y, 0) (Margrabe 1978): V = x N(d1) - y N(d2) with
    sigma^2 = sigma1^2 + sigma2^2 - 2 rho sigma1 sigma2 and
    d1,2 = (ln(x/y) +- sigma^2 tau / 2) / (sigma sqrt(tau)).  Independent of r.

    It solves eq. (bse_change_variable) exactly; at y = 0 it is x, at x = 0 it is 0.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x, y = np.broadcast_arrays(x, y)
    s2 = sigma1 * sigma1 + sigma2 * sigma2 - 2.0 * rho * sigma1 * sigma2
    if tau <= 0.0 or s2 <= 0.0:
        return np.maximum(x - y, 0.0)
    sq = math.sqrt(s2 * tau)
    out = np.zeros(x.shape, dtype=np.float64)
    both = (x > 0.0) & (y > 0.0)
    yzero = (y <= 0.0)
    out[yzero] = x[yzero]
    xb, yb = x[both], y[both]
    d1 = (np.log(xb / yb) + 0.5 * s2 * tau) / sq
    d2 = d1 - sq
    out[both] = xb * ndtr(d1) - yb * ndtr(d2)
    return out


def basket_far_field(x, y, w1, w2, K, r, tau):
    """Far-field value of a basket call: max(w1 x + w2 y - K e^{-r tau}, 0).

    Deep in the money the call is worth its forward, so this is the Dirichlet
    datum on the far edges of the truncated domain (a reading: the paper sets
    Dirichlet data from a closed form, which a basket does not have).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return np.maximum(w1 * x + w2 * y - K * math.exp(-r * tau), 0.0)


def bvn_cdf(h, k, rho):
    """Bivariate standard normal CDF B(h, k; rho) of eq. (solution).

    Written from the integral identity dB/drho = phi2(h, k; rho) (Plackett 1954):
      B(h,k;rho) = N(h) N(k) + int_0^rho exp(-(h^2 - 2 t h k + k^2) / (2 (1 - t^2)))
                                         / (2 pi sqrt(1 - t^2)) dt,
    evaluated with 64-point Gauss-Legendre quadrature in t (|rho| <= 0.9 keeps the
    integrand smooth; that covers every correlation used here).
    """
    h = np.asarray(h, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    h, k = np.broadcast_arrays(h, k)
    if abs(rho) > 0.9:
        raise ValueError("bvn_cdf: |rho| > 0.9 not supported by this quadrature")
    base = ndtr(h) * ndtr(k)
    if rho == 0.0:
        return base
    nodes, weights = np.polynomial.legendre.leggauss(64)
    t = 0.5 * rho * (nodes + 1.0)
    wt = 0.5 * rho * weights
    hh = h[..., None]
    kk = k[..., None]
    one_m = 1.0 - t * t
    f = np.exp(-(hh * hh - 2.0 * t * hh * kk + kk * kk) / (2.0 * one_m)) / (2.0 * math.pi * np.sqrt(one_m))
    return base + np.sum(f * wt, axis=-1)


def cash_or_nothing(x, y, S1, S2, c, r, sigma1, sigma2, rho, tau):
    """Two-asset cash-or-nothing call, eq. (solution): u = c e^{-r tau} B(d_x, d_y; rho),
    d_x = (ln(x/S1) + (r - sigma1^2/2) tau) / (sigma1 sqrt(tau)), same for y.
    At tau = 0 it is the payoff c [x >= S1][y >= S2]; at x = 0 or y = 0 it is 0.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    x, y = np.broadcast_arrays(x, y)
    if tau <= 0.0:
        return np.where((x >= S1) & (y >= S2), c, 0.0)
    out = np.zeros(x.shape, dtype=np.float64)
    pos = (x > 0.0) & (y > 0.0)
    dx = (np.log(x[pos] / S1) + (r - 0.5 * sigma1 ** 2) * tau) / (sigma1 * math.sqrt(tau))
    dy = (np.log(y[pos] / S2) + (r - 0.5 * sigma2 ** 2) * tau) / (sigma2 * math.sqrt(tau))
    out[pos] = c * math.exp(-r * tau) * bvn_cdf(dx, dy, rho)
    return out
