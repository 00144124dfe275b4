"""FP64 forward pass of the Fourier Neural Operator used as the PINO coarse propagator
(Sec. 3.4 lifting / Fourier layers / projection; Sec. 3.5 inputs and outputs).

Test infrastructure only (see ``oracle/__init__``).  numpy.fft is used as a library
primitive for the transforms; everything else is written out here.

Architecture (where the paper leaves the sizes open, the width-32, 12 x 12-mode reading):
  input channels per node: u, x, y, tau_n, dtau, sigma1, sigma2, rho, r      (Sec. 3.5)
  lifting:   v = lift_w^T a + lift_b                        (pointwise, 9 -> width)
  L layers:  v = ReLU( K_l v + pw_w_l^T v + pw_b_l )
             K_l v = irfft2( R_l . rfft2(v) ) keeping ky in [0, my) U [M-my, M) along y and
             kx in [0, mx) of the half spectrum along x; R_l[mode] is a complex width x width
             matrix applied per mode (out[o] = sum_c R[c, o] in[c])
  projection: w = proj2_w . ReLU(proj1_w^T v + proj1_b) + proj2_b   (width -> hidden -> 1)
  output:     u(tau_n + dtau) = u(tau_n) + w  on every node, then the far-field Dirichlet
              data of the payoff at tau_n + dtau on the edges x = xmax and y = ymax.
Arrays are [M][M] with row = y index, column = x index; weights follow
workloads.pino_random_weights.
"""
from __future__ import annotations

import numpy as np

from . import fd
from .resample import bilinear_resample  # noqa: F401  (also used by the FNO tests)


def spectral_conv(v: np.ndarray, R: np.ndarray, mx: int, my: int) -> np.ndarray:
    """K v for v [C][M][M] (real) and R [2*my][mx][C][Co] (complex).

    Row index q of R maps to ky = q for q < my and to ky = M - 2*my + q for q >= my.
    """
    C, M, _ = v.shape
    Co = R.shape[3]
    V = np.fft.rfft2(v, axes=(1, 2))                      # [C][M][M//2 + 1]
    out_hat = np.zeros((Co, M, M // 2 + 1), dtype=np.complex128)
    for q in range(2 * my):
        ky = q if q < my else M - 2 * my + q
        for kx in range(mx):
            out_hat[:, ky, kx] = R[q, kx].T @ V[:, ky, kx]
    return np.fft.irfft2(out_hat, s=(M, M), axes=(1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def input_channels(u, X, Y, tau_n, dtau, params):
    p = params
    M = u.shape[0]
    one = np.ones((M, M))
    return np.stack([u, X, Y, tau_n * one, dtau * one, p.sigma1 * one, p.sigma2 * one,
                     p.rho * one, p.r * one])


def fno_forward(a: np.ndarray, w: dict, mx: int, my: int) -> np.ndarray:
    """Network output w(a) for input channels a [Cin][M][M] (no residual, no boundary)."""
    v = np.einsum("cyx,co->oyx", a, w["lift_w"]) + w["lift_b"][:, None, None]
    L = w["spec_w"].shape[0]
    for l in range(L):
        k = spectral_conv(v, w["spec_w"][l], mx, my)
        pw = np.einsum("cyx,co->oyx", v, w["pw_w"][l]) + w["pw_b"][l][:, None, None]
        v = relu(k + pw)
    h = relu(np.einsum("cyx,ch->hyx", v, w["proj1_w"]) + w["proj1_b"][:, None, None])
    return np.einsum("hyx,h->yx", h, w["proj2_w"]) + w["proj2_b"]


def pino_coarse(u: np.ndarray, xmax: float, tau_n: float, dtau: float, params, w: dict,
                mx: int, my: int, Mp: int = None) -> np.ndarray:
    """One PINO coarse step: u(tau_n) -> u(tau_n + dtau) on an M x M grid.

    The network runs on an Mp x Mp grid (default Mp = M): u is restricted to it bilinearly,
    the network output is prolonged back bilinearly and added to u (reading of the
    resolution change of Sec. 4.4), then the far-field data are set.
    """
    M = u.shape[0]
    Mp = M if Mp is None else Mp
    X, Y = fd.mesh(M, xmax)
    up = u if Mp == M else bilinear_resample(u, Mp)
    Xp, Yp = fd.mesh(Mp, xmax)
    a = input_channels(up, Xp, Yp, tau_n, dtau, params)
    wout = fno_forward(a, w, mx, my)
    if Mp != M:
        wout = bilinear_resample(wout, M)
    out = u + wout
    g = fd.dirichlet(params)(X, Y, tau_n + dtau)
    out[M - 1, :] = g[M - 1, :]
    out[:, M - 1] = g[:, M - 1]
    return out
