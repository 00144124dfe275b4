"""Seeded synthetic workloads for the two-asset Black-Scholes Parareal path.

This module only *describes* inputs: problem sizes, model parameters and seeded
random draws.  It holds none of the method's arithmetic (no stencil, no payoff,
no solver), so both the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2404_02521_gb300``) may import it without sharing any computation.

Payoff codes are the integers of ``include/bsparareal.h``:
0 = basket call max(w1*x + w2*y - K, 0), 1 = exchange max(x - y, 0),
2 = one-asset call max(x - K, 0), 3 = cash-or-nothing (c if x>=S1 and y>=S2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

BASKET, EXCHANGE, CALL1, CASH_OR_NOTHING = 0, 1, 2, 3
COARSE_NUM, COARSE_PINO = 0, 1


@dataclasses.dataclass(frozen=True)
class Params:
    """Model parameters of eq. (bse_change_variable) plus the payoff description."""
    sigma1: float
    sigma2: float
    rho: float
    r: float
    T: float = 1.0
    strike: float = 1.0          # K of the basket / one-asset call; S1 of cash-or-nothing
    w1: float = 0.5
    w2: float = 0.5
    payoff: int = BASKET
    strike2: float = 0.0         # S2 of cash-or-nothing
    cash: float = 1.0            # c of cash-or-nothing


@dataclasses.dataclass(frozen=True)
class Problem:
    """One pricing solve: grid, slices, steps and parameters."""
    name: str
    M: int                 # nodes per axis, x_i = i * xmax / (M - 1)
    xmax: float
    N: int                 # time slices
    fine_steps: int        # implicit-Euler steps per slice for F
    coarse_steps: int      # implicit-Euler steps per slice for the numerical G
    params: Params
    tol: float = 1e-4      # Parareal tolerance (Sec. 4.1 footnote)

    @property
    def dtau_fine(self) -> float:
        return self.params.T / (self.N * self.fine_steps)

    @property
    def dtau_coarse(self) -> float:
        return self.params.T / (self.N * self.coarse_steps)


def basket_cfg1() -> Problem:
    """Basket call, 64x64 on [0,4]^2, N=8, 256 fine and 4 coarse steps per slice."""
    return Problem("basket64", 64, 4.0, 8, 256, 4,
                   Params(0.3, 0.2, 0.5, 0.05, 1.0, 1.0, 0.5, 0.5, BASKET))


def exchange_cfg2(rho: float = 0.7, M: int = 256, N: int = 64, fine_steps: int = 512,
                  coarse_steps: int = 4) -> Problem:
    """Exchange option max(x-y,0) on [0,4]^2 (sigma1=0.25, sigma2=0.35, r=0.03)."""
    return Problem(f"exchange{M}_rho{rho:+.1f}", M, 4.0, N, fine_steps, coarse_steps,
                   Params(0.25, 0.35, rho, 0.03, 1.0, 1.0, 0.5, 0.5, EXCHANGE))


EXCHANGE_RHOS = (-0.5, 0.0, 0.7)


def pino_cfg3(M: int = 128, N: int = 64, fine_steps: int = 512, coarse_steps: int = 4) -> Problem:
    """Basket call on a 128x128 grid, the PINO-Parareal workload."""
    return Problem("basket128", M, 4.0, N, fine_steps, coarse_steps,
                   Params(0.3, 0.2, 0.5, 0.05, 1.0, 1.0, 0.5, 0.5, BASKET))


def large_cfg4(M: int = 1024, N: int = 128, fine_steps: int = 1024,
               coarse_steps: int = 4) -> Problem:
    """Basket call on a 1024x1024 grid, N=128 slices of 1024 fine steps."""
    return Problem("basket1024", M, 4.0, N, fine_steps, coarse_steps,
                   Params(0.3, 0.2, 0.5, 0.05, 1.0, 1.0, 0.5, 0.5, BASKET))


def paper_cash_or_nothing(M: int = 301, N: int = 12, fine_steps: int = 3,
                          coarse_steps: int = 1) -> Problem:
    """The paper's own problem (Sec. 3.2): cash-or-nothing on [0,300]^2, dx=1,
    S1=S2=100, r=1, sigma1=sigma2=0.3, rho=0.5, T=1."""
    return Problem("cash_or_nothing301", M, 300.0, N, fine_steps, coarse_steps,
                   Params(0.3, 0.3, 0.5, 1.0, 1.0, 100.0, 0.5, 0.5, CASH_OR_NOTHING,
                          strike2=100.0, cash=1.0))


# ----------------------------------------------------------------------------------
# Seeded random draws
# ----------------------------------------------------------------------------------

def random_params(rng: np.random.Generator, payoff: int, T: float = 1.0) -> Params:
    """sigma1, sigma2 ~ U[0.1,0.5], rho ~ U[-0.7,0.7], r ~ U[0,0.08]."""
    s1 = float(rng.uniform(0.1, 0.5))
    s2 = float(rng.uniform(0.1, 0.5))
    rho = float(rng.uniform(-0.7, 0.7))
    r = float(rng.uniform(0.0, 0.08))
    return Params(s1, s2, rho, r, T, 1.0, 0.5, 0.5, payoff)


@dataclasses.dataclass(frozen=True)
class Request:
    rid: int
    arrival: float         # seconds after trace start
    problem: Problem


def serving_trace(n_requests: int, rate_per_s: float, seed: int = 12345,
                  grids: Sequence[int] = (64, 128, 256, 512),
                  slices: Sequence[int] = (16, 32, 64),
                  fine_steps: int = 64, coarse_steps: int = 1) -> List[Request]:
    """Poisson arrivals with a 50/50 basket/exchange payoff mix, T ~ U[0.25, 2],
    grid and slice count uniform over the given sets."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s)) if rate_per_s > 0 else 0.0
        payoff = BASKET if rng.uniform() < 0.5 else EXCHANGE
        T = float(rng.uniform(0.25, 2.0))
        p = random_params(rng, payoff, T)
        M = int(rng.choice(np.asarray(grids)))
        N = int(rng.choice(np.asarray(slices)))
        out.append(Request(k, t, Problem(f"req{k}", M, 4.0, N, fine_steps, coarse_steps, p)))
    return out


def random_field(rng: np.random.Generator, M: int, scale: float = 1.0) -> np.ndarray:
    """A seeded smooth-plus-noise [M][M] float64 field (row = y index, column = x index)."""
    g = rng.standard_normal((M, M))
    k = np.linspace(0.0, 1.0, M)
    smooth = np.outer(np.sin(3.0 * k + rng.uniform()), np.cos(2.0 * k + rng.uniform()))
    return scale * (smooth + 0.05 * g)


# ----------------------------------------------------------------------------------
# PINO architecture and seeded weights
# ----------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class PinoArch:
    in_channels: int = 9     # u, x, y, tau_n, dtau, sigma1, sigma2, rho, r
    width: int = 32
    modes_x: int = 12        # kx in [0, modes_x) of the half spectrum along x
    modes_y: int = 12        # ky in [0, modes_y) and [M - modes_y, M) along y
    layers: int = 4
    proj_hidden: int = 128


def pino_random_weights(arch: PinoArch, seed: int = 0, spectral_scale: float = 1.0):
    """Seeded random FNO weights (dict of float64 / complex128 arrays).

    Layout (all row-major):
      lift_w [in_channels][width], lift_b [width]
      spec_w [layers][2*modes_y][modes_x][width_in][width_out]  (complex)
      pw_w   [layers][width_in][width_out], pw_b [layers][width]
      proj1_w [width][proj_hidden], proj1_b [proj_hidden]
      proj2_w [proj_hidden], proj2_b scalar
    """
    rng = np.random.default_rng(seed)
    C, H = arch.width, arch.proj_hidden
    my2 = 2 * arch.modes_y
    s_spec = spectral_scale / (C * C)
    w = {
        "lift_w": rng.standard_normal((arch.in_channels, C)) / math.sqrt(arch.in_channels),
        "lift_b": 0.1 * rng.standard_normal(C),
        "spec_w": s_spec * (rng.uniform(size=(arch.layers, my2, arch.modes_x, C, C))
                            + 1j * rng.uniform(size=(arch.layers, my2, arch.modes_x, C, C))),
        "pw_w": rng.standard_normal((arch.layers, C, C)) / math.sqrt(C),
        "pw_b": 0.1 * rng.standard_normal((arch.layers, C)),
        "proj1_w": rng.standard_normal((C, H)) / math.sqrt(C),
        "proj1_b": 0.1 * rng.standard_normal(H),
        "proj2_w": rng.standard_normal(H) / math.sqrt(H),
        "proj2_b": np.float64(0.0),
    }
    return w
