"""The n-asset generalisation of eq. (fd): centred finite differences of eq. (bse_general) and
implicit Euler, FP64, sparse LU, for any number of assets n (n = 3 gives a 19-point stencil).

Test infrastructure only (see ``oracle/__init__``).  It is the oracle of the n-asset operator
(not yet on the GPU path); for n = 2 it is the scheme of ``oracle/fd.py``.

Operator (eq. bse_general with tau = T - t): u_tau = R u with
  R u = 1/2 sum_{p,q} rho_pq s_p s_q x_p x_q u_{x_p x_q} + r sum_p x_p u_{x_p} - r u,
rho_pp = 1.  The diagonal terms (p = q) are 1/2 s_p^2 x_p^2 u_{x_p x_p}; every pair p < q
appears twice in the double sum, so its term is rho_pq s_p s_q x_p x_q u_{x_p x_q}.
Discretised as eq. (fd) does for n = 2: second differences (u[-1] - 2u[0] + u[+1]) / h^2 along
each axis, the four-point cross difference (u[+p+q] + u[-p-q] - u[+p-q] - u[-p+q]) / (4 h^2)
for each pair, centred first differences (u[+p] - u[-p]) / (2 h).

Grid (reading c2): M nodes per axis including both ends, x_i = i * xmax / (M - 1), the same
spacing h on every axis.  Arrays have shape (M,) * n with axis a holding asset n - a (the
last axis is asset 1, as the column index x of the two-asset arrays [y][x]).

Boundary (reading c3): nodes with some asset index 0 carry the PDE row itself (every term
that would reach index -1 has a coefficient proportional to that asset's x, which is 0);
nodes with some index M - 1 carry Dirichlet data g(x_1, ..., x_n, tau^{m+1}).
"""
from __future__ import annotations

import itertools
from typing import Callable, Dict, Sequence, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BoundaryND = Callable[[Sequence[np.ndarray], float], np.ndarray]


def coords(M: int, xmax: float, n: int):
    """Coordinate arrays (x_1, ..., x_n), each of shape (M,) * n."""
    x = np.arange(M, dtype=np.float64) * (xmax / (M - 1))
    grids = np.meshgrid(*([x] * n), indexing="ij")   # grids[a] varies along axis a
    return [grids[n - 1 - p] for p in range(n)]       # asset p+1 lives on axis n-1-p


def _unit(n: int, p: int, s: int) -> Tuple[int, ...]:
    """Offset (as an axis tuple) of +-1 along asset p (0-based)."""
    off = [0] * n
    off[n - 1 - p] = s
    return tuple(off)


def _add(a: Tuple[int, ...], b: Tuple[int, ...]) -> Tuple[int, ...]:
    return tuple(x + y for x, y in zip(a, b))


def stencil_weights(M: int, xmax: float, sigma: Sequence[float], rho: np.ndarray, r: float
                    ) -> Dict[Tuple[int, ...], np.ndarray]:
    """Weights of R_h at every node, offset (axis tuple) -> array of shape (M,) * n."""
    n = len(sigma)
    X = coords(M, xmax, n)
    h = xmax / (M - 1)
    zero = tuple([0] * n)
    w: Dict[Tuple[int, ...], np.ndarray] = {zero: np.full(X[0].shape, -float(r))}

    def add(off, val):
        w[off] = w.get(off, 0.0) + val

    for p in range(n):
        diff = 0.5 * sigma[p] ** 2 * X[p] ** 2 / h ** 2      # second difference along p
        drift = r * X[p] / (2.0 * h)                         # centred first difference
        add(_unit(n, p, +1), diff + drift)
        add(_unit(n, p, -1), diff - drift)
        add(zero, -2.0 * diff)
    for p, q in itertools.combinations(range(n), 2):
        c = rho[p][q] * sigma[p] * sigma[q] * X[p] * X[q] / (4.0 * h * h)
        add(_add(_unit(n, p, +1), _unit(n, q, +1)), c)
        add(_add(_unit(n, p, -1), _unit(n, q, -1)), c)
        add(_add(_unit(n, p, +1), _unit(n, q, -1)), -c)
        add(_add(_unit(n, p, -1), _unit(n, q, +1)), -c)
    return w


def apply_R(u: np.ndarray, weights) -> np.ndarray:
    """R_h u at the PDE nodes (every index <= M - 2), shape (M - 1,) * n.  Neighbours at index
    -1 only appear with weight zero and are read as 0."""
    n, M = u.ndim, u.shape[0]
    up = np.zeros((M + 1,) * n)
    up[(slice(1, None),) * n] = u
    out = np.zeros((M - 1,) * n)
    core = (slice(0, M - 1),) * n
    for off, wt in weights.items():
        nb = tuple(slice(1 + o, M + o) for o in off)
        out += np.asarray(wt)[core] * up[nb]
    return out


class ImplicitEulerND:
    """(I - dtau R_h) u^{m+1} = u^m on the PDE nodes, Dirichlet data g at the far faces.
    The matrix is assembled once and factorised with sparse LU."""

    def __init__(self, M: int, xmax: float, sigma: Sequence[float], rho, r: float, dtau: float,
                 boundary: BoundaryND):
        self.n, self.M, self.dtau, self.g = len(sigma), M, dtau, boundary
        self.X = coords(M, xmax, self.n)
        n, m = self.n, M - 1
        w = stencil_weights(M, xmax, sigma, np.asarray(rho, dtype=np.float64), r)
        idx = np.indices((m,) * n).reshape(n, -1)             # PDE node indices, axis order
        k = np.ravel_multi_index(idx, (m,) * n)
        rows, cols, vals = [], [], []
        bd_rows, bd_nodes, bd_w = [], [], []
        zero = tuple([0] * n)
        for off, wt in w.items():
            wv = np.asarray(wt)[(slice(0, m),) * n].ravel()
            nb = idx + np.asarray(off).reshape(n, 1)
            neg = (nb < 0).any(axis=0)
            if np.any(wv[neg] != 0.0):
                raise AssertionError("the stencil references index -1 with a nonzero weight")
            inside = ~neg & (nb <= m - 1).all(axis=0)
            far = ~neg & ~inside
            a = -dtau * wv + (1.0 if off == zero else 0.0)
            rows.append(k[inside])
            cols.append(np.ravel_multi_index(nb[:, inside], (m,) * n))
            vals.append(a[inside])
            bd_rows.append(k[far])
            bd_nodes.append(np.ravel_multi_index(nb[:, far], (M,) * n))
            bd_w.append(dtau * wv[far])
        self.A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(m ** n, m ** n))
        self._bd_rows = np.concatenate(bd_rows)
        self._bd_nodes = np.concatenate(bd_nodes)
        self._bd_w = np.concatenate(bd_w)
        self.lu = spla.splu(self.A)

    def step(self, u: np.ndarray, tau_new: float) -> np.ndarray:
        """One implicit-Euler step from u^m (full grid) to tau_new."""
        m = self.M - 1
        gb = np.asarray(self.g(self.X, tau_new), dtype=np.float64)
        rhs = u[(slice(0, m),) * self.n].ravel().copy()
        np.add.at(rhs, self._bd_rows, self._bd_w * gb.ravel()[self._bd_nodes])
        out = gb.copy()
        out[(slice(0, m),) * self.n] = self.lu.solve(rhs).reshape((m,) * self.n)
        return out

    def propagate(self, u: np.ndarray, tau0: float, nsteps: int) -> np.ndarray:
        for s in range(nsteps):
            u = self.step(u, tau0 + (s + 1) * self.dtau)
        return u
