"""Three-asset F (eq. bse_general with n = 3, 19-point stencil) against the n-asset oracle."""
import types

import numpy as np
import pytest

import workloads as wl
from oracle import closed_forms as cf
from oracle import fd_nd
from tests.gpu_util import FP32_FINE_TOL, rel_err

pytestmark = pytest.mark.gpu

XMAX = 4.0
COARSE_TOL = 2e-5   # G against the oracle's exact solves, BiCGSTAB run to 1e-6


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


@pytest.fixture
def tight_g(bs):
    """G's BiCGSTAB solves run to a relative residual of 1e-6 during the test (the oracle's G is
    an exact solve); the library default is 1e-5."""
    bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-6)
    yield
    bs.bs_set_option(bs.OPT_KRYLOV_TOL, 1e-5)


def params3(payoff):
    return types.SimpleNamespace(sigma=(0.3, 0.2, 0.25), rho=(0.5, -0.3, 0.2), r=0.05, strike=1.0,
                                 w=(0.4, 0.35, 0.25), payoff=payoff)


def rho_matrix(p):
    r12, r13, r23 = p.rho
    return np.array([[1.0, r12, r13], [r12, 1.0, r23], [r13, r23, 1.0]])


def oracle_boundary(p):
    if p.payoff == wl.BASKET:
        return lambda X, tau: np.maximum(p.w[0] * X[0] + p.w[1] * X[1] + p.w[2] * X[2]
                                         - p.strike * np.exp(-p.r * tau), 0.0)
    return lambda X, tau: cf.margrabe(X[0], X[1], p.sigma[0], p.sigma[1], p.rho[0], tau)


def oracle_payoff(p, M):
    X = fd_nd.coords(M, XMAX, 3)
    if p.payoff == wl.BASKET:
        return np.maximum(p.w[0] * X[0] + p.w[1] * X[1] + p.w[2] * X[2] - p.strike, 0.0)
    return np.maximum(X[0] - X[1], 0.0)


@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_payoff3(bs, payoff):
    import torch
    p, M = params3(payoff), 13
    u = torch.empty((M, M, M), device="cuda")
    bs.bs_payoff3(M, XMAX, p, u)
    torch.cuda.synchronize()
    np.testing.assert_allclose(u.cpu().double().numpy(), oracle_payoff(p, M), rtol=1e-6, atol=1e-6)


# M = 12 and 21: every node count is ragged against the 256-thread blocks
@pytest.mark.parametrize("M", [12, 21])
@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_fine3_matches_oracle(bs, M, payoff):
    import torch
    p = params3(payoff)
    dtau, nsteps = 0.004, 16
    u0 = oracle_payoff(p, M)
    ie = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, dtau, oracle_boundary(p))
    tau0 = [0.0, 0.1]
    uin = [torch.tensor(u0, dtype=torch.float32, device="cuda") for _ in tau0]
    uout = [torch.empty_like(x) for x in uin]
    bs.fine_propagate3(M, XMAX, p, uin, uout, tau0, dtau, nsteps)
    torch.cuda.synchronize()
    for t, out in zip(tau0, uout):
        want = ie.propagate(u0, t, nsteps)
        assert rel_err(out.cpu().double().numpy(), want) <= FP32_FINE_TOL, (t, M)


def test_fine3_batch_invariance_and_in_place(bs):
    import torch
    p, M = params3(wl.EXCHANGE), 16
    u0 = torch.tensor(oracle_payoff(p, M), dtype=torch.float32, device="cuda")
    one = torch.empty_like(u0)
    bs.fine_propagate3(M, XMAX, p, [u0], [one], [0.05], 0.004, 10)
    many_in = [u0 * 1.5, u0, u0 * 0.5]
    many_out = [torch.empty_like(u0) for _ in many_in]
    bs.fine_propagate3(M, XMAX, p, many_in, many_out, [0.2, 0.05, 0.1], 0.004, 10)
    inplace = u0.clone()
    bs.fine_propagate3(M, XMAX, p, [inplace], [inplace], [0.05], 0.004, 10)
    torch.cuda.synchronize()
    assert torch.equal(one, many_out[1]) and torch.equal(one, inplace)


def serial_fine3(bs, p, M, T, N, fine_steps):
    import torch
    U = torch.empty((N + 1, M, M, M), device="cuda")
    bs.bs_payoff3(M, XMAX, p, U[0])
    sl = T / N
    for n in range(N):
        bs.fine_propagate3(M, XMAX, p, [U[n]], [U[n + 1]], [n * sl], sl / fine_steps, fine_steps)
    torch.cuda.synchronize()
    return U


@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_parareal3_k_equals_n_is_serial_fine(bs, payoff):
    # the Parareal invariant for three assets: K = N reproduces serial fine stepping bitwise
    import torch
    p, M, T, N, fs, cs = params3(payoff), 12, 0.05, 5, 12, 3
    U = torch.empty((N + 1, M, M, M), device="cuda")
    rc, k, defects = bs.parareal_solve3(M, XMAX, p, T, N, fs, cs, 0.0, N, U)
    torch.cuda.synchronize()
    assert rc == 0 and k == N and len(defects) == N
    assert torch.equal(U, serial_fine3(bs, p, M, T, N, fs))


def test_parareal3_matches_oracle_parareal(bs):
    # to tol 1e-4: the oracle's iteration count (exact solves for F and G) and iterate, and
    # within the tolerance of serial fine stepping
    import torch
    from oracle import parareal as opr
    p, M, T, N, fs, cs = params3(wl.BASKET), 12, 0.2, 8, 24, 2
    U = torch.empty((N + 1, M, M, M), device="cuda")
    rc, k, defects = bs.parareal_solve3(M, XMAX, p, T, N, fs, cs, 1e-4, N, U)
    torch.cuda.synchronize()
    sl = T / N
    ieF = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, sl / fs, oracle_boundary(p))
    ieG = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, sl / cs, oracle_boundary(p))
    Uo, ko, do, _ = opr.parareal(oracle_payoff(p, M), lambda u, n: ieF.propagate(u, n * sl, fs),
                                 lambda u, n: ieG.propagate(u, n * sl, cs), N, 1e-4, N)
    assert rc == 0 and k == ko and k < N
    for a, b in zip(defects, do):
        assert abs(a - b) <= 1e-2 * b + 1e-6
    got = U.cpu().double().numpy()
    assert rel_err(got, Uo) <= 1e-4
    serial = serial_fine3(bs, p, M, T, N, fs).cpu().double().numpy()
    assert rel_err(got, serial) <= 1e-3


# steps of 0.1 and 0.025 at M = 12 and 21: Jacobi bounds near 0.8 and above, where the fine
# propagator refuses the step; BiCGSTAB solves them
@pytest.mark.usefixtures("tight_g")
@pytest.mark.parametrize("M,nsteps", [(12, 1), (21, 4)])
@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_coarse3_matches_oracle(bs, M, nsteps, payoff):
    import torch
    p, slice_len, tau0 = params3(payoff), 0.1, 0.05
    u0 = oracle_payoff(p, M)
    ie = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, slice_len / nsteps, oracle_boundary(p))
    uin = torch.tensor(u0, dtype=torch.float32, device="cuda")
    out = torch.empty_like(uin)
    bs.coarse_propagate3(M, XMAX, p, uin, out, tau0, slice_len, nsteps)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().double().numpy(), ie.propagate(u0, tau0, nsteps)) <= COARSE_TOL


def test_coarse3_zero_state_stays_zero(bs):
    # the degenerate case: a zero state under a zero far field (a basket call struck far above
    # the grid) gives b = 0 every step, and the increment must be exactly 0
    import torch
    p, M = params3(wl.BASKET), 12
    p.strike = 1e6                       # the far-field call value is 0 everywhere on the grid
    u = torch.zeros((M, M, M), device="cuda")
    out = torch.full_like(u, 7.0)
    bs.coarse_propagate3(M, XMAX, p, u, out, 0.0, 0.1, 3)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("payoff", [wl.BASKET, wl.EXCHANGE])
def test_parareal3_stiff_coarse_matches_oracle_parareal(bs, payoff):
    # one coarse step per slice of 0.1 (Jacobi bound near 0.8): G by BiCGSTAB at the library
    # default tolerance; the oracle's iteration count, iterate within 1e-4
    import torch
    from oracle import parareal as opr
    p, M, T, N, fs, cs = params3(payoff), 12, 0.4, 4, 25, 1
    U = torch.empty((N + 1, M, M, M), device="cuda")
    rc, k, defects = bs.parareal_solve3(M, XMAX, p, T, N, fs, cs, 1e-4, N, U)
    torch.cuda.synchronize()
    sl = T / N
    ieF = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, sl / fs, oracle_boundary(p))
    ieG = fd_nd.ImplicitEulerND(M, XMAX, p.sigma, rho_matrix(p), p.r, sl / cs, oracle_boundary(p))
    Uo, ko, do, _ = opr.parareal(oracle_payoff(p, M), lambda u, n: ieF.propagate(u, n * sl, fs),
                                 lambda u, n: ieG.propagate(u, n * sl, cs), N, 1e-4, N)
    assert rc == 0 and k == ko
    got = U.cpu().double().numpy()
    assert rel_err(got, Uo) <= 1e-4
