"""Textbook Parareal, eq. (parareal), with the stopping defect of reading c5.

Test infrastructure only (see ``oracle/__init__``).

  u_{n+1}^{k+1} = G(u_n^{k+1}) + F(u_n^k) - G(u_n^k),  n = 0..N-1, k = 0..K-1,
  u_0^k = u_0,  u^0 from one serial sweep of G.

The correction is evaluated as F + (G_new - G_old) (reading c6): when u_n^{k+1}
equals u_n^k bitwise the bracket is exactly zero, so slices that Parareal has
already made exact stay bitwise equal to the serial fine solution.

Defect (reading c5): delta_k = max_n ||u_n^{k+1} - u_n^k||_2 / max_n ||u_n^{k+1}||_2;
the iteration stops once delta_k <= tol or after Kmax iterations.
"""
from __future__ import annotations

from typing import Callable, List

import numpy as np

Prop = Callable[[np.ndarray, int], np.ndarray]


def parareal(u0: np.ndarray, F: Prop, G: Prop, N: int, tol: float, Kmax: int):
    """Run Parareal.  Returns (U [N+1][...], k_done, defects list, history).

    ``history[k]`` is the iterate u^k as an [N+1][...] array (history[0] = the
    coarse sweep).  ``F(u, n)`` and ``G(u, n)`` propagate u over slice n.
    """
    U = [np.array(u0, dtype=np.float64)]
    Gold: List[np.ndarray] = []
    for n in range(N):
        g = G(U[n], n)
        Gold.append(g)
        U.append(g)
    history = [np.stack(U)]
    defects: List[float] = []
    k_done = 0
    for k in range(Kmax):
        Fk = [F(U[n], n) for n in range(N)]           # parallel over slices
        Unew = [U[0]]
        for n in range(N):                             # serial coarse sweep
            gnew = G(Unew[n], n)
            Unew.append(Fk[n] + (gnew - Gold[n]))
            Gold[n] = gnew
        num = max(float(np.linalg.norm((Unew[n] - U[n]).ravel())) for n in range(1, N + 1))
        den = max(float(np.linalg.norm(Unew[n].ravel())) for n in range(1, N + 1))
        delta = num / den if den > 0.0 else num
        U = Unew
        history.append(np.stack(U))
        defects.append(delta)
        k_done = k + 1
        if delta <= tol:
            break
    return np.stack(U), k_done, defects, history


def speedup_bound(P: int, K: int, c_coarse: float, c_fine: float) -> float:
    """Eq. (speedup): S <= 1 / ((1 + K/P) c_coarse/c_fine + K/P)."""
    return 1.0 / ((1.0 + K / P) * (c_coarse / c_fine) + K / P)
