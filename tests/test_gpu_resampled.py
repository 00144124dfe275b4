"""GPU parity of the numerical coarse propagator on a coarser grid with bilinear resampling
(bs_grid_set_coarse) against the FP64 oracle (oracle/resample.py), and of Parareal with it."""
import numpy as np
import pytest

import workloads as wl
from oracle import fd
from oracle import parareal as opr
from oracle import resample as rs
from tests.gpu_util import FP32_FINE_TOL, rel_err, start_state, to_gpu, to_np

pytestmark = pytest.mark.gpu
COARSE_TOL = 2e-5


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


@pytest.fixture
def tight_g(bs):
    """G's BiCGSTAB solves to 1e-6 during the test: the oracle's coarse solves are exact and
    COARSE_TOL is the distance to them at that tolerance."""
    bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-6)
    yield
    bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-5)


@pytest.mark.usefixtures("tight_g")
@pytest.mark.parametrize("M,Mc", [(300, 100), (256, 64), (129, 65), (512, 256)])
def test_resampled_coarse_matches_oracle(bs, M, Mc):
    import torch
    p = wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE)
    u0 = start_state(M, 4.0, p, "payoff")
    g = bs.Grid(M, 4.0)
    g.set_coarse(Mc)
    uin = to_gpu(u0)
    out = torch.empty_like(uin)
    bs.coarse_propagate(g, bs.COARSE_NUM, None, p, uin, out, 0.25, 1.0 / 64, 4)
    torch.cuda.synchronize()
    want = rs.resampled_coarse(u0.astype(np.float64), 4.0, p, 0.25, 1.0 / 64, 4, Mc)
    assert rel_err(to_np(out), want) <= COARSE_TOL


@pytest.mark.usefixtures("tight_g")
def test_parareal_with_resampled_coarse(bs):
    import torch
    pb = wl.Problem("rs128", 128, 4.0, 8, 256, 2, wl.basket_cfg1().params)
    Mc = 64
    g = bs.Grid(pb.M, pb.xmax)
    g.set_coarse(Mc)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    rc, k, defects = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                       None, 1e-4, pb.N, U)
    torch.cuda.synchronize()
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
    G = rs.ResampledPropagator(pb.M, pb.xmax, pb.params, pb.N, pb.coarse_steps, Mc)
    serial = fd.serial_fine(pb)
    Uo, ko, do, _ = opr.parareal(serial[0], F, G, pb.N, 1e-4, pb.N)
    assert rc == 0 and k == ko
    assert rel_err(to_np(U), Uo) <= 3 * COARSE_TOL
    for a, b in zip(defects, do):
        assert abs(a - b) <= 1e-3 * b + 1e-6
    assert rel_err(to_np(U), serial) <= 1e-3
    # K = N reproduces serial fine stepping whatever G is
    rc, k, _ = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps, None,
                                 0.0, pb.N, U)
    torch.cuda.synchronize()
    assert k == pb.N and rel_err(to_np(U), serial) <= FP32_FINE_TOL


def test_set_coarse_rejects_bad_sizes(bs):
    g = bs.Grid(64, 4.0)
    with pytest.raises(bs.BSError):
        g.set_coarse(4)
    with pytest.raises(bs.BSError):
        g.set_coarse(65)
    g.set_coarse(64)   # same grid: plain coarse propagation
    g.set_coarse(0)


@pytest.mark.parametrize("M,Mc,N", [(300, 100, 8), (128, 64, 12)])
def test_pipelined_resampled_equals_phase_driver(bs, M, Mc, N):
    # F chunks overlapped with the chunked coarse sweep on the coarse grid: every slice's
    # coarse solve starts afresh, so the iteration is the phase-by-phase driver's bit for bit --
    # to convergence, and after two fixed iterations, where an F chunk that read its first
    # state after the next sweep had rewritten it would show in slice 3
    import torch
    pb = wl.Problem("rsp", M, 4.0, N, 64 if M == 128 else 96, 2, wl.basket_cfg1().params)
    g = bs.Grid(pb.M, pb.xmax)
    g.set_coarse(Mc)
    for tol, K in ((1e-4, pb.N), (0.0, 2), (0.0, 3)):
        out = []
        for pipe in (0, 1):
            U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
            try:
                bs.bs_set_option(bs.OPT_PIPELINE, pipe)
                rc, k, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                             None, tol, K, U)
                torch.cuda.synchronize()
            finally:
                bs.bs_set_option(bs.OPT_PIPELINE, 1)
            out.append((rc, k, d, U))
        assert out[0][1] == out[1][1] and out[0][0] == out[1][0], (tol, K)
        assert (out[0][0] == 0) if K == pb.N else (out[0][1] == K)
        assert out[0][2] == out[1][2], (tol, K)
        assert torch.equal(out[0][3], out[1][3]), (tol, K)
