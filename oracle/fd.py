"""Eq. (fd): centred 9-point finite differences + implicit Euler, FP64, sparse LU.

Test infrastructure only (see ``oracle/__init__``).

Grid (reading c2): M nodes per axis including both ends, x_i = i * xmax / (M - 1),
y_j likewise, dx = dy.  Arrays are [M][M] with row = j (y index) and column = i
(x index).

Operator (eq. bse_change_variable, tau = T - t): u_tau = R u with
  R u = 1/2 s1^2 x^2 u_xx + 1/2 s2^2 y^2 u_yy + rho s1 s2 x y u_xy + r x u_x + r y u_y - r u,
discretised by eq. (fd): second differences (u[i-1] - 2u[i] + u[i+1]) / dx^2, the
four-point cross difference (u[i+1,j+1] + u[i-1,j-1] - u[i+1,j-1] - u[i-1,j+1]) /
(4 dx dy) and centred first differences (u[i+1] - u[i-1]) / (2 dx).

Implicit Euler: (u^{n+1} - u^n) / dtau - R_h u^{n+1} = 0, i.e. (I - dtau R_h) u^{n+1} = u^n.

Boundary (reading c3): rows i = 0 and j = 0 are the PDE row itself (its x- or
y-coefficients vanish there, so no ghost node is referenced); the far edges
i = M-1 and j = M-1 carry Dirichlet data g(x, y, tau^{n+1}).
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import closed_forms as cf

BASKET, EXCHANGE, CALL1, CASH_OR_NOTHING = 0, 1, 2, 3

BoundaryFn = Callable[[np.ndarray, np.ndarray, float], np.ndarray]


def nodes(M: int, xmax: float) -> np.ndarray:
    """x_i = i * xmax / (M - 1), i = 0..M-1 (reading c2)."""
    return np.arange(M, dtype=np.float64) * (xmax / (M - 1))


def mesh(M: int, xmax: float):
    x = nodes(M, xmax)
    X, Y = np.meshgrid(x, x, indexing="xy")      # X[j, i] = x_i, Y[j, i] = y_j
    return X, Y


def payoff(params, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Terminal payoff u(tau = 0) for the payoff code of ``params``."""
    p = params
    if p.payoff == BASKET:
        return np.maximum(p.w1 * X + p.w2 * Y - p.strike, 0.0)
    if p.payoff == EXCHANGE:
        return np.maximum(X - Y, 0.0)
    if p.payoff == CALL1:
        return np.maximum(X - p.strike, 0.0)
    if p.payoff == CASH_OR_NOTHING:
        # Sec. 3.2: c if x >= S1 and y >= S2, else 0
        return np.where((X >= p.strike) & (Y >= p.strike2), p.cash, 0.0)
    raise ValueError(f"unknown payoff {p.payoff}")


def dirichlet(params) -> BoundaryFn:
    """Far-field Dirichlet data g(x, y, tau) for the payoff of ``params`` (reading c3)."""
    p = params
    if p.payoff == BASKET:
        return lambda X, Y, tau: cf.basket_far_field(X, Y, p.w1, p.w2, p.strike, p.r, tau)
    if p.payoff == EXCHANGE:
        return lambda X, Y, tau: cf.margrabe(X, Y, p.sigma1, p.sigma2, p.rho, tau)
    if p.payoff == CALL1:
        return lambda X, Y, tau: cf.bs_call_1d(X, p.strike, p.r, p.sigma1, tau) + 0.0 * Y
    if p.payoff == CASH_OR_NOTHING:
        return lambda X, Y, tau: cf.cash_or_nothing(X, Y, p.strike, p.strike2, p.cash, p.r,
                                                     p.sigma1, p.sigma2, p.rho, tau)
    raise ValueError(f"unknown payoff {p.payoff}")


def stencil_weights(M: int, xmax: float, sigma1: float, sigma2: float, rho: float, r: float):
    """Weights of R_h at every node, as a dict offset (di, dj) -> [M][M] array.

    Collected from eq. (fd) term by term:
      diffusion in x: 1/2 s1^2 x_i^2 / dx^2 on (-1,0), (+1,0); -2x that on (0,0)
      diffusion in y: 1/2 s2^2 y_j^2 / dy^2 on (0,-1), (0,+1); -2x that on (0,0)
      cross:          rho s1 s2 x_i y_j / (4 dx dy) on (+1,+1), (-1,-1); minus on (+1,-1), (-1,+1)
      drift:          r x_i / (2 dx) on (+1,0), minus on (-1,0); r y_j / (2 dy) on (0,+1), minus on (0,-1)
      reaction:       -r on (0,0)
    """
    X, Y = mesh(M, xmax)
    dx = xmax / (M - 1)
    dy = dx
    dxx = 0.5 * sigma1 ** 2 * X ** 2 / dx ** 2
    dyy = 0.5 * sigma2 ** 2 * Y ** 2 / dy ** 2
    cxy = rho * sigma1 * sigma2 * X * Y / (4.0 * dx * dy)
    drx = r * X / (2.0 * dx)
    dry = r * Y / (2.0 * dy)
    w = {
        (0, 0): -2.0 * dxx - 2.0 * dyy - r,
        (-1, 0): dxx - drx,
        (+1, 0): dxx + drx,
        (0, -1): dyy - dry,
        (0, +1): dyy + dry,
        (+1, +1): cxy.copy(),
        (-1, -1): cxy.copy(),
        (+1, -1): -cxy,
        (-1, +1): -cxy,
    }
    return w


def apply_R(u: np.ndarray, weights) -> np.ndarray:
    """R_h u at the nodes 0 <= i, j <= M-2 (the rows that carry a PDE equation).

    Returns an [M-1][M-1] array.  Neighbours at i = -1 or j = -1 only appear with
    weight zero (the coefficients vanish at x = 0, y = 0), so they are read as 0.
    """
    M = u.shape[0]
    up = np.zeros((M + 1, M + 1))
    up[1:, 1:] = u                   # up[j+1, i+1] = u[j, i]; index -1 -> 0
    out = np.zeros((M - 1, M - 1))
    for (di, dj), w in weights.items():
        nb = up[1 + dj: M + dj, 1 + di: M + di]
        out += w[: M - 1, : M - 1] * nb
    return out


class ImplicitEuler:
    """(I - dtau R_h) u^{n+1} = u^n on the unknowns 0 <= i, j <= M-2, Dirichlet at the
    far edges.  The matrix is assembled once and factorised with sparse LU."""

    def __init__(self, M: int, xmax: float, params, dtau: float,
                 boundary: Optional[BoundaryFn] = None):
        self.M, self.xmax, self.p, self.dtau = M, xmax, params, dtau
        self.g = boundary if boundary is not None else dirichlet(params)
        self._builtin_g = boundary is None
        self.X, self.Y = mesh(M, xmax)
        n = M - 1
        w = stencil_weights(M, xmax, params.sigma1, params.sigma2, params.rho, params.r)
        rows, cols, vals = [], [], []
        # Dirichlet couplings: (unknown index, boundary j, boundary i, weight)
        self._bd_rows, self._bd_j, self._bd_i, self._bd_w = [], [], [], []
        J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        k = (J * n + I).ravel()
        for (di, dj), wt in w.items():
            wv = wt[:n, :n].ravel()
            ii = (I + di).ravel()
            jj = (J + dj).ravel()
            a = -dtau * wv + (1.0 if (di, dj) == (0, 0) else 0.0)
            inside = (ii >= 0) & (jj >= 0) & (ii <= n - 1) & (jj <= n - 1)
            neg = (ii < 0) | (jj < 0)
            if np.any(wv[neg] != 0.0):
                raise AssertionError("eq. (fd) references a node left of x=0 with nonzero weight")
            rows.append(k[inside]); cols.append((jj * n + ii)[inside]); vals.append(a[inside])
            far = (~inside) & (~neg)
            self._bd_rows.append(k[far]); self._bd_j.append(jj[far]); self._bd_i.append(ii[far])
            self._bd_w.append(dtau * wv[far])
        self.A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(n * n, n * n))
        self._bd_rows = np.concatenate(self._bd_rows)
        self._bd_j = np.concatenate(self._bd_j)
        self._bd_i = np.concatenate(self._bd_i)
        self._bd_w = np.concatenate(self._bd_w)
        self.lu = spla.splu(self.A)

    def boundary_values(self, tau: float) -> np.ndarray:
        """g at time tau; only the far edges i = M-1 and j = M-1 are used.  The built-in
        closed forms act elementwise and are evaluated on those edges alone (the rest of the
        returned grid is zero); a caller's boundary function gets the whole grid."""
        if not self._builtin_g:
            return np.asarray(self.g(self.X, self.Y, tau), dtype=np.float64)
        M = self.M
        out = np.zeros((M, M), dtype=np.float64)
        out[M - 1, :] = np.asarray(self.g(self.X[M - 1, :], self.Y[M - 1, :], tau), dtype=np.float64)
        out[:, M - 1] = np.asarray(self.g(self.X[:, M - 1], self.Y[:, M - 1], tau), dtype=np.float64)
        return out

    def step(self, u: np.ndarray, tau_new: float) -> np.ndarray:
        """One implicit-Euler step from u^n (full [M][M] grid) to tau_new."""
        M, n = self.M, self.M - 1
        gb = self.boundary_values(tau_new)
        rhs = u[:n, :n].ravel().copy()
        np.add.at(rhs, self._bd_rows, self._bd_w * gb[self._bd_j, self._bd_i])
        sol = self.lu.solve(rhs)
        out = gb.copy()
        out[:n, :n] = sol.reshape(n, n)
        return out

    def propagate(self, u: np.ndarray, tau0: float, nsteps: int) -> np.ndarray:
        for m in range(nsteps):
            u = self.step(u, tau0 + (m + 1) * self.dtau)
        return u


def initial_state(M: int, xmax: float, params) -> np.ndarray:
    """u(tau = 0): the payoff on the grid."""
    X, Y = mesh(M, xmax)
    return payoff(params, X, Y)


class SlicePropagator:
    """F or the numerical G of Sec. 3.1: ``steps`` implicit-Euler steps over slice n
    of a problem with N slices on [0, T] (reading c4: dtau = T / (N * steps))."""

    def __init__(self, M: int, xmax: float, params, N: int, steps: int,
                 boundary: Optional[BoundaryFn] = None):
        self.N, self.steps = N, steps
        self.slice_len = params.T / N
        self.ie = ImplicitEuler(M, xmax, params, self.slice_len / steps, boundary)

    def __call__(self, u: np.ndarray, n: int) -> np.ndarray:
        return self.ie.propagate(u, n * self.slice_len, self.steps)


def serial_fine(problem, boundary: Optional[BoundaryFn] = None):
    """Serial fine solution U_n = F^n(u_0), n = 0..N, as an [N+1][M][M] array."""
    F = SlicePropagator(problem.M, problem.xmax, problem.params, problem.N,
                        problem.fine_steps, boundary)
    u = initial_state(problem.M, problem.xmax, problem.params)
    out = [u]
    for n in range(problem.N):
        u = F(u, n)
        out.append(u)
    return np.stack(out)


def jacobi_contraction(M: int, xmax: float, params, dtau: float) -> float:
    """max over PDE rows of sum_k |offdiag_k| / |diag| of I - dtau R_h (the Gershgorin
    bound on the Jacobi iteration matrix; < 1 means Jacobi contracts in the max norm)."""
    w = stencil_weights(M, xmax, params.sigma1, params.sigma2, params.rho, params.r)
    n = M - 1
    diag = 1.0 - dtau * w[(0, 0)][:n, :n]
    off = sum(np.abs(dtau * wt[:n, :n]) for key, wt in w.items() if key != (0, 0))
    return float(np.max(off / np.abs(diag)))
