"""The paper's own problem (Sec. 3.2): two-asset cash-or-nothing call on [0,300]^2 with
dx = dy = 1 (301 x 301 nodes), r = 1, sigma1 = sigma2 = 0.3, rho = 0.5, T = 1, N = 10
slices.  The expected values come from tests/golden/cash_or_nothing301.json, written by
tests/golden/make_paper_golden.py from the FP64 oracle alone."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import FP32_FINE_TOL, to_np

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "cash_or_nothing301.json")) as f:
        return json.load(f)


def problem(gd):
    return wl.paper_cash_or_nothing(N=gd["N"], fine_steps=gd["fine_steps"])


def check_against_golden(U, gd, tol):
    rows, cols = np.array(gd["rows"]), np.array(gd["cols"])
    worst = 0.0
    for key, vals in gd["slices"].items():
        got = to_np(U[int(key)])[rows, cols]
        worst = max(worst, np.max(np.abs(got - np.array(vals))) / gd["maxabs"][key])
    assert worst <= tol, worst
    return worst


def test_serial_fine_matches_oracle(bs, golden):
    import torch
    pb = problem(golden)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, U[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [U[n]], [U[n + 1]], [n * sl], [pb.dtau_fine], pb.fine_steps)
    torch.cuda.synchronize()
    check_against_golden(U, golden, FP32_FINE_TOL)


@pytest.mark.parametrize("coarse_steps", [1, 4])
def test_parareal_converges_to_the_fine_solution(bs, golden, coarse_steps):
    # numerical G with the paper's coarse step 0.1 (one step per slice) or four steps.  A
    # coarse step of 0.1 on this grid is very stiff (dtau sigma^2 i^2 ~ 800 at the far edge),
    # so its BiCGSTAB solves get a larger iteration cap.
    import torch
    pb = problem(golden)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    try:
        bs.bs_set_option(bs.OPT_KRYLOV_MAXIT, 20000)
        rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, coarse_steps,
                                           None, 1e-4, pb.N, U)
        torch.cuda.synchronize()
    finally:
        bs.bs_set_option(bs.OPT_KRYLOV_MAXIT, 400)
    # with 1536 fine steps per slice, one coarse step of 0.1 is a poor approximation of F and
    # Parareal needs most of its N = 10 iterations; four coarse steps converge in a few
    assert rc == 0 and k <= (9 if coarse_steps == 1 else 4), (rc, k, defects)
    assert all(b < a for a, b in zip(defects, defects[1:]))   # monotone defects (Fig. 3 shape)
    check_against_golden(U, golden, 1e-3)


def test_paper_step_sizes_serial_fine_matches_oracle(bs):
    # serial fine stepping with the paper's three substeps per 0.1-slice (Sec. 4.1): every step
    # is too large for Jacobi sweeps, so F solves it by BiCGSTAB; held to the FP32 fine bound
    # at the golden's sampled nodes of slices 1, 2, 5 and 10 (eq. fd, implicit Euler)
    import torch
    with open(os.path.join(HERE, "golden", "cash_or_nothing301_paper_steps.json")) as f:
        gd = json.load(f)
    pb = wl.paper_cash_or_nothing(N=gd["N"], fine_steps=gd["fine_steps"])
    g = bs.Grid(pb.M, pb.xmax)
    assert bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine) == 0
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, U[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [U[n]], [U[n + 1]], [n * sl], [pb.dtau_fine],
                                  pb.fine_steps)
    torch.cuda.synchronize()
    assert not bs.bs_grid_stats(g)[1]
    check_against_golden(U, gd, FP32_FINE_TOL)


def test_paper_step_sizes_parareal_matches_oracle(bs):
    # the paper's configuration: three fine substeps per 0.1-slice and one coarse step
    # (Sec. 4.1).  Both are too large for Jacobi sweeps on this grid, so F and G are BiCGSTAB
    # solves; the GPU Parareal takes the oracle's iteration count and defects.  The oracle's G
    # is an exact solve, so G's solves run to 1e-6 here: at the default 1e-5 the iteration
    # count is the same but on this very stiff coarse step (dtau sigma^2 i^2 ~ 800) the
    # smallest defect moves by 10%.
    import torch
    with open(os.path.join(HERE, "golden", "cash_or_nothing301_paper_steps.json")) as f:
        gd = json.load(f)
    pb = wl.paper_cash_or_nothing(N=gd["N"], fine_steps=gd["fine_steps"])
    g = bs.Grid(pb.M, pb.xmax)
    assert bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine) == 0
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    try:
        bs.bs_set_option(bs.OPT_KRYLOV_MAXIT, 20000)
        bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-6)
        rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, 1, None, 1e-4,
                                           pb.N, U)
        torch.cuda.synchronize()
    finally:
        bs.bs_set_option(bs.OPT_KRYLOV_MAXIT, 400)
        bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-5)
    assert rc == 0 and k == gd["parareal_k"]
    for a, b in zip(defects, gd["parareal_defects"]):
        assert abs(a - b) <= 2e-2 * b + 1e-6
    rows, cols = np.array(gd["rows"]), np.array(gd["cols"])
    got = to_np(U[pb.N])[rows, cols]
    assert np.max(np.abs(got - np.array(gd["parareal_final"]))) <= 2e-4
