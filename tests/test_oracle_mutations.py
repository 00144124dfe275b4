"""Planted mistakes in the oracle's stencil (on the CPU) must fail its pins.

Each mutation is a plausible slip in writing eq. (fd): a flipped cross-term sign,
a swapped drift direction, a dropped reaction term, transposed volatilities or a
cross term missing its factor.  The biquadratic-exactness pin must reject each.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import fd
from tests.test_oracle_fd import PARAM_SETS, continuous_R_monomial


def biquadratic_error(weights_fn, p, M=9, xmax=4.0):
    X, Y = fd.mesh(M, xmax)
    w = weights_fn(M, xmax, p.sigma1, p.sigma2, p.rho, p.r)
    worst = 0.0
    for a in range(3):
        for b in range(3):
            u = X ** a * Y ** b
            want = continuous_R_monomial(p, a, b) * u[: M - 1, : M - 1]
            worst = max(worst, float(np.max(np.abs(fd.apply_R(u, w) - want))))
    return worst


def mutate(kind):
    def sw(M, xmax, s1, s2, rho, r):
        if kind == "swap_sigma":
            s1, s2 = s2, s1
        w = fd.stencil_weights(M, xmax, s1, s2, rho, r)
        if kind == "cross_sign":
            for k in [(1, 1), (-1, -1), (1, -1), (-1, 1)]:
                w[k] = -w[k]
        elif kind == "drift_sign":
            w[(1, 0)], w[(-1, 0)] = w[(-1, 0)], w[(1, 0)]
        elif kind == "drop_reaction":
            w[(0, 0)] = w[(0, 0)] + r
        elif kind == "cross_half":
            for k in [(1, 1), (-1, -1), (1, -1), (-1, 1)]:
                w[k] = 0.5 * w[k]
        elif kind == "y_drift_transposed":
            w[(0, 1)], w[(0, -1)] = w[(0, -1)], w[(0, 1)]
        return w
    return sw


def test_unmutated_passes():
    for p in PARAM_SETS:
        assert biquadratic_error(fd.stencil_weights, p) < 1e-9


@pytest.mark.parametrize("kind", ["cross_sign", "drift_sign", "drop_reaction", "swap_sigma",
                                  "cross_half", "y_drift_transposed"])
def test_mutation_is_caught(kind):
    p = wl.Params(0.3, 0.2, 0.5, 0.05)
    assert biquadratic_error(mutate(kind), p) > 1e-3
