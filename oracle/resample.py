"""Bilinear resampling between node grids and the numerical coarse propagator on a coarser
grid (the resolution change of Sec. 4.4 applied to the numerical coarse model of Sec. 3.2).

Test infrastructure only (see ``oracle/__init__``).

Reading: for a state u on M x M nodes and a coarse grid of Mc x Mc nodes on the same domain,
    G(u) = P( G_c(R u) ),   far-field data at tau_n + dtau_slice,
where R and P are bilinear interpolation at node positions (both grids include both ends)
and G_c takes csteps implicit-Euler steps of eq. (fd) on the coarse grid (sparse LU).  The
coarse state is prolonged (spatially coarsened Parareal): fine-scale components of u, which
F damps within a slice, are dropped by G too.  Prolonging only the coarse increment and
keeping u's fine detail would pass those components through G undamped, and Parareal then
stalls (defects grow over the first iterations on the exchange-option workload).  With
Mc = M, R and P are identities and G is the plain coarse propagation.
"""
from __future__ import annotations

import numpy as np

from . import fd


def bilinear_resample(u: np.ndarray, M_out: int) -> np.ndarray:
    """Bilinear interpolation of a node-based field on [0, xmax]^2 from M_in to M_out nodes
    per axis (both grids include both ends): node j of the output sits at j*(M_in-1)/(M_out-1)
    in input index units."""
    M_in = u.shape[0]
    t = np.arange(M_out) * (M_in - 1) / (M_out - 1)
    i0 = np.minimum(np.floor(t).astype(int), M_in - 2)
    f = t - i0
    rows = u[i0, :] * (1 - f)[:, None] + u[i0 + 1, :] * f[:, None]
    return rows[:, i0] * (1 - f)[None, :] + rows[:, i0 + 1] * f[None, :]


def resampled_coarse(u: np.ndarray, xmax: float, params, tau_n: float, dtau_slice: float,
                     csteps: int, Mc: int, boundary=None, ie=None) -> np.ndarray:
    """G(u) for one slice (see the module docstring); ie: a prebuilt fd.ImplicitEuler on the
    coarse grid with step dtau_slice / csteps."""
    M = u.shape[0]
    if ie is None:
        ie = fd.ImplicitEuler(Mc, xmax, params, dtau_slice / csteps, boundary)
    uc = u if Mc == M else bilinear_resample(u, Mc)
    gc = ie.propagate(uc, tau_n, csteps)
    out = gc if Mc == M else bilinear_resample(gc, M)
    g = (boundary if boundary is not None else fd.dirichlet(params))
    X, Y = fd.mesh(M, xmax)
    gb = np.asarray(g(X, Y, tau_n + dtau_slice), dtype=np.float64)
    out[M - 1, :] = gb[M - 1, :]
    out[:, M - 1] = gb[:, M - 1]
    return out


class ResampledPropagator:
    """Slice map n -> G(u) with the resampled numerical coarse model (for oracle Parareal)."""

    def __init__(self, M: int, xmax: float, params, N: int, csteps: int, Mc: int, boundary=None):
        self.xmax, self.p, self.N, self.csteps, self.Mc = xmax, params, N, csteps, Mc
        self.slice = params.T / N
        self.boundary = boundary
        self.ie = fd.ImplicitEuler(Mc, xmax, params, self.slice / csteps, boundary)

    def __call__(self, u: np.ndarray, n: int) -> np.ndarray:
        return resampled_coarse(u, self.xmax, self.p, n * self.slice, self.slice, self.csteps, self.Mc,
                                self.boundary, self.ie)
