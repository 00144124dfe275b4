"""FP64 physics-informed loss of a predicted slice (Sec. 3.5, eq. bs_totalloss: the PDE term).

Test infrastructure only (see ``oracle/__init__``).

A coarse propagator maps u(tau_n) to a prediction u~ of u(tau_n + dtau).  The PDE term of the
training loss measures how far u~ is from satisfying eq. (bse_change_variable) over the slice,
discretised by eq. (fd) with the slice as one implicit-Euler step.  The collocation points are
the nodes that carry a PDE row, 0 <= i, j <= M-2 (reading c3; the far edges hold Dirichlet
data):

  r = (u~ - u_prev) / dtau - R_h u~          at every collocation point,
  loss = (1 / n) sum r^2,                     n = (M - 1)^2,
  d loss / d u~ = (2 / n) (E^T r / dtau - R_h^T r),

where E places the collocation points into the full [M][M] grid and R_h^T r is R_h's
adjoint applied to r (written out below as a scatter of each row's weights).
"""
from __future__ import annotations

import numpy as np

from . import fd


def residual(u_pred: np.ndarray, u_prev: np.ndarray, dtau: float, weights) -> np.ndarray:
    """r at the collocation points, an [M-1][M-1] array."""
    M = u_pred.shape[0]
    n = M - 1
    return (u_pred[:n, :n] - u_prev[:n, :n]) / dtau - fd.apply_R(u_pred, weights)


def loss(u_pred: np.ndarray, u_prev: np.ndarray, dtau: float, weights) -> float:
    r = residual(u_pred, u_prev, dtau, weights)
    return float(np.mean(r * r))


def loss_grad(u_pred: np.ndarray, u_prev: np.ndarray, dtau: float, weights) -> np.ndarray:
    """d loss / d u_pred on the full [M][M] grid.

    Each collocation point p contributes 2 r_p / n times d r_p / d u~: 1 / dtau at p itself and
    -w_o(p) at the node p + o for every stencil offset o (the weight with which row p reads
    that node).  Offsets that leave the grid at x = 0 or y = 0 carry weight zero.
    """
    M = u_pred.shape[0]
    n = M - 1
    r = residual(u_pred, u_prev, dtau, weights)
    c = 2.0 * r / (n * n)
    g = np.zeros((M, M))
    g[:n, :n] += c / dtau
    J, I = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for (di, dj), w in weights.items():
        wv = w[:n, :n]
        tj, ti = J + dj, I + di
        ok = (tj >= 0) & (ti >= 0)
        if np.any(wv[~ok] != 0.0):
            raise AssertionError("eq. (fd) reads a node left of x = 0 or below y = 0 with nonzero weight")
        np.add.at(g, (tj[ok], ti[ok]), -(c * wv)[ok])
    return g
