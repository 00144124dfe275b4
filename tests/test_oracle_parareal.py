"""Pins for the Parareal oracle (oracle/parareal.py), eq. (parareal) and eq. (speedup)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fd
from oracle import parareal as pr


def small_problem(payoff=wl.BASKET, N=6):
    p = wl.Params(0.3, 0.2, 0.5, 0.05, payoff=payoff)
    return wl.Problem("small", 17, 4.0, N, 12, 2, p)


def props(pb):
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
    G = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.coarse_steps)
    return F, G


@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_k_equals_n_reproduces_serial_fine_bitwise(payoff):
    pb = small_problem(payoff)
    F, G = props(pb)
    serial = fd.serial_fine(pb)
    U, k, defects, hist = pr.parareal(serial[0], F, G, pb.N, tol=0.0, Kmax=pb.N)
    assert k == pb.N
    assert np.array_equal(U, serial)


def test_exact_prefix_after_k_iterations():
    # u_n^k = F^n(u_0) bitwise for n <= k (F + (G_new - G_old) with a zero bracket)
    pb = small_problem()
    F, G = props(pb)
    serial = fd.serial_fine(pb)
    _, _, _, hist = pr.parareal(serial[0], F, G, pb.N, tol=0.0, Kmax=pb.N)
    for k, Uk in enumerate(hist):
        assert np.array_equal(Uk[: k + 1], serial[: k + 1]), k


def test_coarse_equal_fine_converges_in_one_iteration():
    pb = small_problem()
    F, _ = props(pb)
    serial = fd.serial_fine(pb)
    U, k, defects, _ = pr.parareal(serial[0], F, F, pb.N, tol=1e-14, Kmax=pb.N)
    assert k == 1 and defects[0] == 0.0
    assert np.array_equal(U, serial)


def test_tolerance_reached_and_error_small():
    pb = wl.basket_cfg1()
    pb = wl.Problem(pb.name, 33, pb.xmax, pb.N, 64, pb.coarse_steps, pb.params)
    F, G = props(pb)
    serial = fd.serial_fine(pb)
    U, k, defects, _ = pr.parareal(serial[0], F, G, pb.N, tol=1e-4, Kmax=pb.N)
    assert defects[-1] <= 1e-4 and k < pb.N
    # defect is monotone on this problem (observed, not a theorem)
    assert all(defects[i + 1] < defects[i] for i in range(len(defects) - 1))
    assert np.max(np.abs(U - serial)) / np.max(np.abs(serial)) < 1e-3


def test_speedup_bound():
    # eq. (speedup) and its two limits
    s = pr.speedup_bound(64, 2, 2.2, 350.0)
    assert s <= min(350.0 / 2.2, 64 / 2)
    assert abs(pr.speedup_bound(10 ** 9, 1, 1.0, 100.0) - 100.0) < 1e-4
    assert abs(pr.speedup_bound(64, 2, 0.0, 1.0) - 32.0) < 1e-12
