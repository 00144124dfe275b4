"""GPU parity of the PINO coarse propagator (tensor-core BF16 FNO, Sec. 3.4-3.5) against the
FP64 oracle forward of the same weights, and Parareal with the PINO as G."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import fd
from oracle import fno
from tests.gpu_util import FP32_FINE_TOL, rel_err, start_state, to_gpu, to_np

pytestmark = pytest.mark.gpu

# BF16 operands (unit roundoff 2^-9) pass through about 30 rounded contractions between the
# input and the network output (6 per Fourier layer, 4 layers, lifting and projection); with
# FP32 accumulation the output error stays within a few percent of the output's magnitude.
PINO_REL_TOL = 4e-2


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


@pytest.fixture(scope="module")
def weights(tmp_path_factory):
    from paper_2404_02521_gb300 import pino_io
    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=11, spectral_scale=8.0)
    path = str(tmp_path_factory.mktemp("pino") / "w.bin")
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y,
                          arch.layers, arch.proj_hidden)
    w2, _ = pino_io.read_weights(path)   # the float32 values the library loads
    return path, w2, arch


def network_grid(M):
    return 128 if M <= 128 else 256


@pytest.mark.parametrize("M,payoff", [(128, wl.BASKET), (256, wl.EXCHANGE), (96, wl.EXCHANGE),
                                      (200, wl.BASKET), (64, wl.BASKET), (1024, wl.BASKET)])
def test_pino_step_matches_oracle(bs, weights, M, payoff):
    import torch
    path, w, arch = weights
    net = bs.Pino(path)
    p = wl.basket_cfg1().params if payoff == wl.BASKET else wl.exchange_cfg2(-0.5).params
    u0 = start_state(M, 4.0, p, "random", seed=M)
    g = bs.Grid(M, 4.0)
    uin = to_gpu(u0)
    out = torch.empty_like(uin)
    tau0, dtau = 0.25, 1.0 / 64
    bs.coarse_propagate(g, bs.COARSE_PINO, net, p, uin, out, tau0, dtau, 1)
    torch.cuda.synchronize()
    want = fno.pino_coarse(u0.astype(np.float64), 4.0, tau0, dtau, p, w, arch.modes_x,
                           arch.modes_y, Mp=network_grid(M))
    got = to_np(out)
    d_got, d_want = got - u0, want - u0.astype(np.float64)
    err = float(np.max(np.abs(d_got - d_want)) / np.max(np.abs(d_want)))
    print(f"M={M}: network-output rel. err {err:.3e}")
    assert err <= PINO_REL_TOL
    # far-field edges are the closed form exactly as on the fine path
    assert np.max(np.abs(got[M - 1] - want[M - 1])) < 1e-5 * (1 + np.max(np.abs(want)))


def test_pino_parareal_invariants(bs, weights):
    # Parareal with any coarse model reproduces serial fine after N iterations (bitwise), and
    # the first k+1 slices are exact after k iterations.
    import torch
    path, _, _ = weights
    net = bs.Pino(path)
    pb = wl.Problem("pino128", 128, 4.0, 4, 1024, 1, wl.basket_cfg1().params)
    g = bs.Grid(pb.M, pb.xmax)
    S = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, S[0])
    sl = pb.params.T / pb.N
    for n in range(pb.N):
        bs.fine_propagate_batched(g, [pb.params], [S[n]], [S[n + 1]], [n * sl],
                                  [sl / pb.fine_steps], pb.fine_steps)
    U = torch.empty_like(S)
    rc, k, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_PINO, 1, net, 0.0,
                                 pb.N, U)
    torch.cuda.synchronize()
    assert k == pb.N and torch.equal(U, S)
    for K in (1, 2):
        rc, k, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_PINO, 1, net,
                                     0.0, K, U)
        torch.cuda.synchronize()
        assert torch.equal(U[: K + 1], S[: K + 1])
    assert rel_err(to_np(S), fd.serial_fine(pb)) <= FP32_FINE_TOL


def test_pino_parareal_matches_oracle_parareal(bs, tmp_path):
    # GPU PINO-Parareal (eq. parareal with the BF16 tensor-core FNO as G) beside the textbook
    # FP64 Parareal of the oracle with the FP64 FNO forward of the same weights, three
    # iterations on 64 x 64 states (the network runs on its 128 x 128 grid: restriction and
    # prolongation are part of G).  The projection weights are scaled down so that G is the
    # identity plus a small network increment w, as a trained coarse model is.
    import torch
    from paper_2404_02521_gb300 import pino_io
    from oracle import parareal as opr
    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=23, spectral_scale=8.0)
    w["proj2_w"] = 0.05 * w["proj2_w"]
    w["proj2_b"] = np.float64(0.0)
    path = str(tmp_path / "w.bin")
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y,
                          arch.layers, arch.proj_hidden)
    w32, _ = pino_io.read_weights(path)
    net = bs.Pino(path)
    pb = wl.Problem("pino64", 64, 4.0, 4, 128, 1, wl.basket_cfg1().params)   # Jacobi bound 0.6
    K = 3
    g = bs.Grid(pb.M, pb.xmax)
    sl = pb.params.T / pb.N
    Ug, dg = [], None
    for k in range(K + 1):
        U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
        rc, kd, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_PINO, 1, net,
                                      0.0, k, U)
        torch.cuda.synchronize()
        assert kd == k
        Ug.append(to_np(U))
        dg = d
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)

    def G(u, n):
        return fno.pino_coarse(u, pb.xmax, n * sl, sl, pb.params, w32, arch.modes_x, arch.modes_y, Mp=128)

    # the network increments on the GPU's inputs bound the BF16 error of one G evaluation
    Gv = [[G(Ug[k][n], n) for n in range(pb.N)] for k in range(K + 1)]
    wmax = max(float(np.max(np.abs(Gv[k][n] - Ug[k][n]))) for k in range(K + 1) for n in range(pb.N))
    vmax = float(np.max(np.abs(Ug[K])))
    eps_g = PINO_REL_TOL * wmax
    # the initial sweep: u_{n+1}^0 = G(u_n^0)
    for n in range(pb.N):
        assert np.max(np.abs(Ug[0][n + 1] - Gv[0][n])) <= eps_g + FP32_FINE_TOL * vmax, n
    # every iterate, slice by slice: u_{n+1}^k = F(u_n^{k-1}) + G(u_n^k) - G(u_n^{k-1}) on the
    # GPU's own previous iterates, within two network errors and the FP32 fine bound
    for k in range(1, K + 1):
        assert np.array_equal(Ug[k][0], Ug[0][0])
        for n in range(pb.N):
            want = F(Ug[k - 1][n], n) + (Gv[k][n] - Gv[k - 1][n])
            err = float(np.max(np.abs(Ug[k][n + 1] - want)))
            assert err <= 2 * eps_g + FP32_FINE_TOL * vmax, (k, n, err / wmax)
    # the defects are those of the GPU iterates (reading c5; the GPU sums squares in FP32 per
    # block of 256 nodes and over blocks in FP64)
    for k in range(1, K + 1):
        num = max(float(np.linalg.norm(Ug[k][n] - Ug[k - 1][n])) for n in range(1, pb.N + 1))
        den = max(float(np.linalg.norm(Ug[k][n])) for n in range(1, pb.N + 1))
        assert abs(dg[k - 1] - num / den) <= 1e-4 * num / den, k
    # against the oracle's own PINO-Parareal: each iterate is a chain of at most 2N + 1 network
    # evaluations (and fine propagations, which do not amplify), so it stays within that many
    # network errors; the defects agree to the same relative accuracy
    u0 = Ug[0][0].astype(np.float64)
    _, _, do, hist = opr.parareal(u0, F, G, pb.N, 0.0, K)
    for k in range(K + 1):
        err = float(np.max(np.abs(Ug[k] - hist[k])))
        assert err <= (2 * pb.N + 1) * eps_g + FP32_FINE_TOL * vmax, (k, err / wmax)
    for a, b in zip(dg, do):
        assert abs(a - b) <= (2 * pb.N + 1) * PINO_REL_TOL * b, (a, b)


@pytest.mark.parametrize("M,B", [(96, 5), (128, 3), (64, 130)])
def test_pino_batched_equals_single(bs, weights, M, B):
    # several states through one network launch chain (B = 130: two chunks of at most 128)
    # give each state's single-state result bit for bit
    import torch
    path, _, _ = weights
    net = bs.Pino(path)
    rng = np.random.default_rng(M + B)
    ps = [wl.random_params(rng, wl.BASKET if b % 2 else wl.EXCHANGE) for b in range(B)]
    ins = [to_gpu(start_state(M, 4.0, ps[b], "random", seed=b)) for b in range(B)]
    outs = [torch.empty_like(u) for u in ins]
    taus = [0.01 * b for b in range(B)]
    g = bs.Grid(M, 4.0)
    bs.coarse_propagate_batched(g, bs.COARSE_PINO, net, ps, ins, outs, taus, 1.0 / 64)
    torch.cuda.synchronize()
    for b in sorted({0, 1, B // 2, B - 1}):
        one = torch.empty_like(ins[b])
        bs.coarse_propagate(g, bs.COARSE_PINO, net, ps[b], ins[b], one, taus[b], 1.0 / 64, 1)
        torch.cuda.synchronize()
        assert torch.equal(one, outs[b]), b


def test_pino_load_rejects_bad_files(bs, tmp_path):
    p = tmp_path / "bad.bin"
    p.write_bytes(b"BSPINO01" + b"\0" * 16)
    with pytest.raises(bs.BSError):
        bs.Pino(str(p))
    q = tmp_path / "short.bin"
    from paper_2404_02521_gb300 import pino_io
    arch = wl.PinoArch(width=8, modes_x=2, modes_y=2, layers=1, proj_hidden=16)
    pino_io.write_weights(str(q), wl.pino_random_weights(arch), 9, 8, 2, 2, 1, 16)
    q.write_bytes(q.read_bytes()[:-4])
    with pytest.raises(bs.BSError):
        bs.Pino(str(q))
