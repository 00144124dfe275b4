"""Full-size checks in the launch configurations the benchmark times: the exchange-option
workload (256x256 on [0,4]^2, N=64 slices of 512 fine steps, sigma1=0.25, sigma2=0.35,
r=0.03, T=1) and the large single solve (basket on 1024x1024, N=128 slices of 1024 fine
steps, numerical G on 256x256).

The expected values come from tests/golden/exchange256_rho*.json, written by
tests/golden/make_exchange256_golden.py (sampled nodes after slices 1, 2, 8, 32, 64 of the
serial fine solution), and tests/golden/basket1024_slice0.json, written by
tests/golden/make_basket1024_golden.py (sampled nodes after 16, 128 and 1024 fine steps of
the large solve's first slice), both from the FP64 oracle alone.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import closed_forms as cf
from oracle import fd
from tests.gpu_util import FP32_FINE_TOL, to_np

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


def golden(rho):
    with open(os.path.join(HERE, "golden", f"exchange256_rho{rho:+.1f}.json")) as f:
        return json.load(f)


def gpu_serial(bs, pb):
    import torch
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, U[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [U[n]], [U[n + 1]], [n * sl], [pb.dtau_fine],
                                  pb.fine_steps)
    torch.cuda.synchronize()
    return g, U


@pytest.mark.parametrize("rho", wl.EXCHANGE_RHOS)
def test_serial_fine_matches_oracle_golden(bs, rho):
    gd = golden(rho)
    pb = wl.exchange_cfg2(rho)
    _, U = gpu_serial(bs, pb)
    rows, cols = np.array(gd["rows"]), np.array(gd["cols"])
    for key, vals in gd["slices"].items():
        got = to_np(U[int(key)])[rows, cols]
        err = np.max(np.abs(got - np.array(vals))) / gd["maxabs"][key]
        assert err <= FP32_FINE_TOL, (key, err)


@pytest.mark.parametrize("rho", wl.EXCHANGE_RHOS)
def test_parareal_converges_to_serial_fine(bs, rho):
    # the configuration of the benchmark: tol 1e-4, numerical coarse model, 4 steps/slice
    import torch
    gd = golden(rho)
    pb = wl.exchange_cfg2(rho)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM,
                                       pb.coarse_steps, None, pb.tol, pb.N, U)
    torch.cuda.synchronize()
    assert rc == 0 and defects[-1] <= pb.tol and k <= 4
    rows, cols = np.array(gd["rows"]), np.array(gd["cols"])
    got = to_np(U[pb.N])[rows, cols]
    # a converged iterate differs from the fine solution by about the last defect
    assert np.max(np.abs(got - np.array(gd["slices"]["64"]))) / gd["maxabs"]["64"] <= 3 * pb.tol
    # Margrabe closed form on the interior, within the discretisation error of the grid
    X, Y = fd.mesh(pb.M, pb.xmax)
    ex = cf.margrabe(X, Y, pb.params.sigma1, pb.params.sigma2, rho, pb.params.T)
    box = (X >= 1.0) & (X <= 3.0) & (Y >= 1.0) & (Y <= 3.0)
    assert np.max(np.abs(to_np(U[pb.N]) - ex)[box]) < 2e-3


def test_k_equals_n_full_size_bitwise(bs):
    import torch
    pb = wl.exchange_cfg2(0.7)
    _, S = gpu_serial(bs, pb)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty_like(S)
    rc, k, _ = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM,
                                 pb.coarse_steps, None, 0.0, pb.N, U)
    torch.cuda.synchronize()
    assert k == pb.N
    assert torch.equal(U, S)


def golden1024():
    with open(os.path.join(HERE, "golden", "basket1024_slice0.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("nsteps", [16, 128, 1024])
def test_large_solve_fine_slice_matches_oracle_golden(bs, nsteps):
    # F of the large solve's first slice from the payoff, batched with three more states as in
    # Parareal's fine launches (temporally blocked tiles): the cold first step, the extrapolated
    # steps and the late steps of the sweep schedule, against the FP64 oracle's sampled nodes
    import torch
    gd = golden1024()
    pb = wl.large_cfg4()
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((4, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, U[0])
    U[1:].copy_(U[0].expand(3, pb.M, pb.M))
    F = torch.empty_like(U)
    sl = pb.params.T / pb.N
    bs.fine_propagate_batched(g, [pb.params] * 4, list(U), list(F), [0.0, sl, 2 * sl, 3 * sl],
                              [pb.dtau_fine] * 4, nsteps)
    torch.cuda.synchronize()
    rows, cols = np.array(gd["rows"]), np.array(gd["cols"])
    got = to_np(F[0])[rows, cols]
    err = np.max(np.abs(got - np.array(gd["steps"][str(nsteps)]))) / gd["maxabs"][str(nsteps)]
    assert err <= FP32_FINE_TOL, err


def test_large_solve_converges_to_serial_fine(bs):
    # the benchmark's large solve: Parareal to tol 1e-4 converges and its u_N is within the
    # tolerance of serial fine stepping on the same GPU
    import torch
    pb = wl.large_cfg4()
    g = bs.Grid(pb.M, pb.xmax)
    g.set_coarse(256)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                       None, pb.tol, pb.N, U)
    torch.cuda.synchronize()
    assert rc == 0 and defects[-1] <= pb.tol and k < pb.N
    S = torch.empty((2, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, S[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [S[n % 2]], [S[(n + 1) % 2]], [n * sl], [pb.dtau_fine],
                                  pb.fine_steps)
    torch.cuda.synchronize()
    assert float((U[pb.N] - S[pb.N % 2]).abs().max() / S[pb.N % 2].abs().max()) <= 10 * pb.tol
