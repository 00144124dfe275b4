"""Degenerate cases of the Parareal iteration and the largest grid (GB300).

- one slice: the first correction makes the slice exact, so k = 1 and the result is serial
  fine stepping bitwise;
- Kmax = 0: only the initial coarse sweep runs, and U is the serial coarse propagation;
- the largest grid bs_grid_create accepts (4096^2): K = N reproduces serial fine stepping
  bitwise, a property that holds at any size and needs no oracle solve.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import fd
from tests.gpu_util import FP32_FINE_TOL, rel_err, to_np

pytestmark = pytest.mark.gpu

COARSE_TOL = 2e-5   # G against the oracle's exact solves, BiCGSTAB run to 1e-6


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


def parareal(bs, pb, tol, Kmax):
    import torch
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                       None, tol, Kmax, U)
    torch.cuda.synchronize()
    return rc, k, defects, U


def serial_fine_gpu(bs, pb):
    import torch
    g = bs.Grid(pb.M, pb.xmax)
    S = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, S[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [S[n]], [S[n + 1]], [n * sl], [pb.dtau_fine], pb.fine_steps)
    torch.cuda.synchronize()
    return S


@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_single_slice_is_fine_stepping(bs, payoff):
    import torch
    base = wl.basket_cfg1().params if payoff == wl.BASKET else wl.exchange_cfg2(0.7).params
    pb = wl.Problem("one-slice", 64, 4.0, 1, 64, 2, base)
    rc, k, defects, U = parareal(bs, pb, 1e-4, 1)
    assert rc == 0 and k == 1
    assert torch.equal(U, serial_fine_gpu(bs, pb))
    assert rel_err(to_np(U[1]), fd.serial_fine(pb)[1]) <= FP32_FINE_TOL


def test_kmax_zero_is_the_coarse_sweep(bs):
    # no iteration: U_n = G^n(u_0), the serial coarse propagation, with status MAXITER
    pb = wl.Problem("coarse-only", 64, 4.0, 6, 64, 2, wl.basket_cfg1().params)
    try:
        bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-6)
        rc, k, defects, U = parareal(bs, pb, 1e-4, 0)
    finally:
        bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-5)
    assert rc == bs._lib.BS_ERR_MAXITER and k == 0 and defects == []
    G = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.coarse_steps)
    u = fd.initial_state(pb.M, pb.xmax, pb.params)
    want = [u]
    for n in range(pb.N):
        u = G(u, n)
        want.append(u)
    assert rel_err(to_np(U), np.stack(want)) <= COARSE_TOL


def test_largest_grid_k_equals_n(bs):
    # 4096^2 nodes: cluster-tile F and the global-memory coarse solver.  A short horizon keeps
    # the fine steps on Jacobi (q < 0.8 needs dtau ~ 1e-7 at this many nodes) and the coarse
    # solves easy; K = N must still reproduce serial fine stepping bitwise.
    import torch
    p = wl.Params(0.05, 0.04, 0.5, 0.01, T=2e-6, payoff=wl.EXCHANGE)
    pb = wl.Problem("largest", 4096, 4.0, 2, 8, 1, p)
    g = bs.Grid(pb.M, pb.xmax)
    assert bs.bs_fine_sweeps(g, p, pb.dtau_fine) > 0
    rc, k, defects, U = parareal(bs, pb, 0.0, pb.N)
    assert k == pb.N
    S = serial_fine_gpu(bs, pb)
    assert bool(torch.isfinite(U).all())
    assert torch.equal(U, S)
