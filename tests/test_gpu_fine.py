"""GPU parity of the fine propagator F (fine_propagate_batched, eq. fd + implicit Euler)
against the FP64 sparse-LU oracle, element by element."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import (FP32_FINE_TOL, dtau_for, oracle_fine, rel_err, start_state, to_gpu,
                            to_np)

pytestmark = pytest.mark.gpu

PARAMS = [
    wl.Params(0.3, 0.2, 0.5, 0.05, payoff=wl.BASKET),
    wl.Params(0.25, 0.35, -0.5, 0.03, payoff=wl.EXCHANGE),
    wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE),
    wl.Params(0.4, 0.15, 0.0, 0.08, strike=1.2, payoff=wl.CALL1),
]


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


# M spans one CTA (33, 64), two bands with a ragged tail (100), 7 bands with padding (200)
# and the full 8-CTA cluster (256).
@pytest.mark.parametrize("M", [5, 33, 64, 100, 128, 200, 256])
@pytest.mark.parametrize("pi", range(len(PARAMS)))
def test_fine_matches_oracle(bs, M, pi):
    import torch
    p = PARAMS[pi]
    xmax = 4.0
    dtau = dtau_for(M, p)
    nsteps = 12 if M >= 200 else 30
    u0 = start_state(M, xmax, p, "payoff" if pi % 2 == 0 else "random", seed=M)
    tau0 = 0.05 * pi
    g = bs.Grid(M, xmax)
    uin = to_gpu(u0)
    uout = torch.empty_like(uin)
    bs.fine_propagate_batched(g, [p], [uin], [uout], [tau0], [dtau], nsteps)
    torch.cuda.synchronize()
    want = oracle_fine(M, xmax, p, u0, tau0, dtau, nsteps)
    assert rel_err(to_np(uout), want) <= FP32_FINE_TOL


@pytest.mark.parametrize("M,pi", [(300, 0), (300, 2), (512, 1)])
def test_fine_tiles_match_oracle(bs, M, pi):
    # grids beyond one cluster: one implicit step per launch over haloed tiles
    import torch
    p = PARAMS[pi]
    xmax = 4.0
    dtau = dtau_for(M, p)
    nsteps = 6
    u0 = start_state(M, xmax, p, "random" if pi else "payoff", seed=M)
    g = bs.Grid(M, xmax)
    uin = to_gpu(u0)
    uout = torch.empty_like(uin)
    bs.fine_propagate_batched(g, [p, p], [uin, uin], [uout, torch.empty_like(uin)], [0.1, 0.1],
                              [dtau, dtau], nsteps)
    one = uin.clone()
    bs.fine_propagate_batched(g, [p], [one], [one], [0.1], [dtau], 1)    # in place, one step
    torch.cuda.synchronize()
    want = oracle_fine(M, xmax, p, u0, 0.1, dtau, nsteps)
    assert rel_err(to_np(uout), want) <= FP32_FINE_TOL
    assert rel_err(to_np(one), oracle_fine(M, xmax, p, u0, 0.1, dtau, 1)) <= FP32_FINE_TOL


@pytest.fixture
def tile_layout(bs):
    """Force the fine tiles' region layout (1: 256 x 256 regions, 2: 288 x 288) for a test."""
    def force(k):
        bs.bs_set_option(bs.OPT_FINE_TILE, k)
    yield force
    bs.bs_set_option(bs.OPT_FINE_TILE, 0)


@pytest.mark.parametrize("layout", [1, 2])
@pytest.mark.parametrize("M,pi,nsteps", [(300, 1, 40), (301, 2, 40), (516, 0, 24)])
def test_tile_temporal_blocking_matches_oracle(bs, tile_layout, M, pi, nsteps, layout):
    # several whole implicit steps per tile launch (the halo grows with the launch's sweeps):
    # long enough to reach the late two- and three-sweep steps; M = 301 runs the 4-byte copy
    # path (M not a multiple of 4), M = 300 and 516 the 16-byte one; both region layouts
    import torch
    tile_layout(layout)
    p = PARAMS[pi]
    dtau = dtau_for(M, p)
    u0 = start_state(M, 4.0, p, "random", seed=M + nsteps)
    g = bs.Grid(M, 4.0)
    uin = to_gpu(u0)
    out = torch.empty_like(uin)
    bs.fine_propagate_batched(g, [p], [uin], [out], [0.05], [dtau], nsteps)
    inplace = uin.clone()
    bs.fine_propagate_batched(g, [p], [inplace], [inplace], [0.05], [dtau], nsteps)
    torch.cuda.synchronize()
    assert torch.equal(out, inplace)
    assert rel_err(to_np(out), oracle_fine(M, 4.0, p, u0, 0.05, dtau, nsteps)) <= FP32_FINE_TOL


@pytest.mark.parametrize("M,pi,nsteps", [(300, 0, 40), (301, 1, 30), (516, 2, 24), (1024, 0, 20)])
def test_tile_layouts_agree_bitwise(bs, tile_layout, M, pi, nsteps):
    # the two region layouts (256 x 256 regions and up to 24 sweeps per launch, 288 x 288 and up
    # to 16) compute every node of a region's exact part with the same operations in the same
    # order from its global indices, and a launch boundary carries the state exactly, so they
    # agree bit for bit though their launches and tiles differ
    import torch
    p = PARAMS[pi]
    dtau = dtau_for(M, p)
    u0 = to_gpu(start_state(M, 4.0, p, "random", seed=7 * M))
    g = bs.Grid(M, 4.0)
    outs = []
    for layout in (1, 2):
        tile_layout(layout)
        out = torch.empty_like(u0)
        bs.fine_propagate_batched(g, [p, p], [u0, u0], [out, torch.empty_like(u0)], [0.0, 0.1],
                                  [dtau, dtau / 2], nsteps)
        torch.cuda.synchronize()
        outs.append(out)
    assert torch.equal(outs[0], outs[1])


def test_tile_step_split_over_launches(bs):
    # the cold first step needs more sweeps than one tile launch's halo holds: it runs as
    # two launches (the first leaves the increment unapplied); an item with fewer sweeps in
    # the same batch is copied through the extra launch
    import torch
    M, xmax = 300, 4.0
    p = PARAMS[0]
    g = bs.Grid(M, xmax)
    lo, hi = 1e-6, 1e-2
    for _ in range(60):           # step with 36..48 cold sweeps (Jacobi bound still < 0.8)
        mid = (lo * hi) ** 0.5
        m0 = bs.bs_fine_sweeps(g, p, mid, first_step=True)
        if m0 == 0 or m0 > 48:
            hi = mid
        elif m0 < 36:
            lo = mid
        else:
            break
    dtau = mid
    assert 32 < bs.bs_fine_sweeps(g, p, dtau, first_step=True) <= 48
    small = dtau / 16
    assert bs.bs_fine_sweeps(g, p, small, first_step=True) <= 32
    u0 = start_state(M, xmax, p, "payoff")
    uin = to_gpu(u0)
    outs = [torch.empty_like(uin) for _ in range(2)]
    bs.fine_propagate_batched(g, [p, p], [uin, uin], outs, [0.1, 0.1], [dtau, small], 3)
    one = uin.clone()
    bs.fine_propagate_batched(g, [p], [one], [one], [0.1], [dtau], 1)
    torch.cuda.synchronize()
    assert rel_err(to_np(outs[0]), oracle_fine(M, xmax, p, u0, 0.1, dtau, 3)) <= FP32_FINE_TOL
    assert rel_err(to_np(outs[1]), oracle_fine(M, xmax, p, u0, 0.1, small, 3)) <= FP32_FINE_TOL
    assert rel_err(to_np(one), oracle_fine(M, xmax, p, u0, 0.1, dtau, 1)) <= FP32_FINE_TOL


@pytest.mark.parametrize("M", [129, 200, 256])
def test_band_layouts_agree_bitwise(bs, tile_layout, M):
    # a state in one cluster of 8 CTAs of 32 rows or of 16 CTAs of 16 rows: the same
    # operations per node, so the same result bit for bit, one state or several per launch
    import torch
    p = PARAMS[1]
    dtau = dtau_for(M, p)
    u0 = to_gpu(start_state(M, 4.0, p, "random", seed=3 * M))
    g = bs.Grid(M, 4.0)
    outs = {}
    for layout in (1, 2):
        tile_layout(layout)
        for n in (1, 3):
            out = [torch.empty_like(u0) for _ in range(n)]
            bs.fine_propagate_batched(g, [p] * n, [u0] * n, out, [0.05 * k for k in range(n)], [dtau] * n, 40)
            torch.cuda.synchronize()
            outs[(layout, n)] = out[0]
    tile_layout(0)
    auto = torch.empty_like(u0)
    bs.fine_propagate_batched(g, [p], [u0], [auto], [0.0], [dtau], 40)
    torch.cuda.synchronize()
    for key, out in outs.items():
        assert torch.equal(out, outs[(1, 1)]), key
    assert torch.equal(auto, outs[(1, 1)])


@pytest.mark.parametrize("layout", [1, 2])
def test_tile_one_sweep_commit_in_split_step(bs, tile_layout, layout):
    # items of one batch with different step sizes: the batch's cold step takes 26 sweeps and
    # runs as two launches of 13, and item B's takes 14, so B's step ends one sweep into the
    # second launch -- a piece that forms b from hi and commits the step.  B equals its
    # propagation alone bit for bit, and both items the oracle (both region layouts)
    import torch
    tile_layout(layout)
    M, xmax = 300, 4.0
    p = PARAMS[0]
    g = bs.Grid(M, xmax)

    def dtau_with(m):
        lo, hi = 1e-7, 1e-2
        for _ in range(80):
            mid = (lo * hi) ** 0.5
            k = bs.bs_fine_sweeps(g, p, mid, first_step=True)
            if k == m:
                return mid
            if k == 0 or k > m:
                hi = mid
            else:
                lo = mid
        raise AssertionError(f"no step size with {m} cold sweeps")

    dA, dB = dtau_with(26), dtau_with(14)
    u0 = start_state(M, xmax, p, "random", seed=5)
    uin = to_gpu(u0)
    outs = [torch.empty_like(uin) for _ in range(2)]
    bs.fine_propagate_batched(g, [p, p], [uin, uin], outs, [0.1, 0.1], [dA, dB], 3)
    alone = torch.empty_like(uin)
    bs.fine_propagate_batched(g, [p], [uin], [alone], [0.1], [dB], 3)
    torch.cuda.synchronize()
    assert torch.equal(outs[1], alone)
    assert rel_err(to_np(outs[1]), oracle_fine(M, xmax, p, u0, 0.1, dB, 3)) <= FP32_FINE_TOL
    assert rel_err(to_np(outs[0]), oracle_fine(M, xmax, p, u0, 0.1, dA, 3)) <= FP32_FINE_TOL


def test_tile_batch_composition_invariance(bs):
    # a tile item's result does not depend on the halo width chosen for its batch (the
    # halo follows the largest sweep count in the launch)
    import torch
    M = 300
    pA = wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE)
    pB = wl.Params(0.45, 0.3, -0.3, 0.06, payoff=wl.BASKET)
    g = bs.Grid(M, 4.0)
    u0 = to_gpu(start_state(M, 4.0, pA, "random", seed=3))
    dA = 1.0 / 65536
    for dB, nsteps in ((1.0 / 65536, 1), (1.0 / 16384, 3)):
        a = torch.empty_like(u0)
        bs.fine_propagate_batched(g, [pA], [u0], [a], [0.1], [dA], nsteps)
        ab = [torch.empty_like(u0) for _ in range(2)]
        bs.fine_propagate_batched(g, [pA, pB], [u0, u0], ab, [0.1, 0.2], [dA, dB], nsteps)
        torch.cuda.synchronize()
        assert bs.bs_fine_sweeps(g, pB, dB, True) > bs.bs_fine_sweeps(g, pA, dA, True)
        assert torch.equal(a, ab[0])


def test_batch_invariance_and_in_place(bs):
    import torch
    M, xmax = 100, 4.0
    items = [(PARAMS[0], 0.0), (PARAMS[1], 0.3), (PARAMS[3], 0.1), (PARAMS[2], 0.7)]
    dt = [dtau_for(M, p) for p, _ in items]
    u0 = [start_state(M, xmax, p, "payoff") for p, _ in items]
    g = bs.Grid(M, xmax)
    ins = [to_gpu(u) for u in u0]
    outs = [torch.empty_like(x) for x in ins]
    bs.fine_propagate_batched(g, [p for p, _ in items], ins, outs, [t for _, t in items], dt, 9)
    alone = torch.empty_like(ins[1])
    bs.fine_propagate_batched(g, [items[1][0]], [ins[1]], [alone], [items[1][1]], [dt[1]], 9)
    inplace = ins[2].clone()
    bs.fine_propagate_batched(g, [items[2][0]], [inplace], [inplace], [items[2][1]], [dt[2]], 9)
    torch.cuda.synchronize()
    assert torch.equal(alone, outs[1])
    assert torch.equal(inplace, outs[2])
    for (p, t0), u, o, d in zip(items, u0, outs, dt):
        assert rel_err(to_np(o), oracle_fine(M, xmax, p, u, t0, d, 9)) <= FP32_FINE_TOL


def test_zero_steps_is_a_copy(bs):
    import torch
    g = bs.Grid(40, 4.0)
    u = to_gpu(np.random.default_rng(1).uniform(size=(40, 40)))
    out = torch.zeros_like(u)
    bs.fine_propagate_batched(g, [PARAMS[0]], [u], [out], [0.0], [1e-4], 0)
    torch.cuda.synchronize()
    assert torch.equal(out, u)


def test_large_batch_spans_several_launches(bs):
    import torch
    M, xmax, n = 33, 4.0, 100     # more items than one launch's descriptor table
    p = PARAMS[1]
    dt = dtau_for(M, p)
    g = bs.Grid(M, xmax)
    u0 = start_state(M, xmax, p, "payoff")
    ins = [to_gpu(u0) for _ in range(n)]
    outs = [torch.empty_like(x) for x in ins]
    taus = [0.01 * k for k in range(n)]
    bs.fine_propagate_batched(g, [p] * n, ins, outs, taus, [dt] * n, 5)
    torch.cuda.synchronize()
    for k in (0, 57, 99):
        assert rel_err(to_np(outs[k]), oracle_fine(M, xmax, p, u0, taus[k], dt, 5)) <= FP32_FINE_TOL


def test_long_chain_compensated_state(bs):
    # 4096 steps on a 64-grid: without the compensated (hi, lo) state, increments below
    # half an ulp would be lost and the error would exceed the FP32 bound.
    import torch
    M, xmax = 64, 4.0
    p = wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE)
    dtau, nsteps = 1.0 / 4096, 4096
    u0 = start_state(M, xmax, p, "payoff")
    g = bs.Grid(M, xmax)
    uin = to_gpu(u0)
    out = torch.empty_like(uin)
    bs.fine_propagate_batched(g, [p], [uin], [out], [0.0], [dtau], nsteps)
    torch.cuda.synchronize()
    assert rel_err(to_np(out), oracle_fine(M, xmax, p, u0, 0.0, dtau, nsteps)) <= FP32_FINE_TOL


def test_bad_step_is_rejected(bs):
    g = bs.Grid(64, 4.0)
    u = to_gpu(np.zeros((64, 64)))
    with pytest.raises(bs.BSError):
        bs.fine_propagate_batched(g, [PARAMS[0]], [u], [u], [0.0], [-1e-3], 3)
    with pytest.raises(bs.BSError):
        bs.fine_propagate_batched(g, [PARAMS[0]], [u], [u], [0.0], [0.0], 3)


# BiCGSTAB stops each step at a relative residual of 1e-6 of the Jacobi-scaled system
# (BS_OPT_FINE_KRYLOV_TOL); F by BiCGSTAB steps is held to the FP32 fine bound like the Jacobi
# steps (measured: at most 5.6e-7 of max|V| on these cases).
KRYLOV_TOL = FP32_FINE_TOL


@pytest.mark.parametrize("M,pi", [(64, 1), (100, 0), (300, 2)])
def test_krylov_fine_matches_oracle(bs, M, pi):
    # steps whose Jacobi bound is >= 0.8 are solved by BiCGSTAB, one cluster per state; two
    # states with different start times share a batched launch, a third with other
    # parameters gets its own
    import torch
    p, q = PARAMS[pi], PARAMS[(pi + 1) % len(PARAMS)]
    dtau = 1.0 / 256
    g = bs.Grid(M, 4.0)
    assert bs.bs_fine_sweeps(g, p, dtau) == 0 and bs.bs_fine_sweeps(g, q, dtau) == 0
    u0 = start_state(M, 4.0, p, "payoff")
    uin = to_gpu(u0)
    outs = [torch.empty_like(uin) for _ in range(3)]
    bs.fine_propagate_batched(g, [p, p, q], [uin, uin, uin], outs, [0.1, 0.3, 0.1], [dtau] * 3, 3)
    torch.cuda.synchronize()
    for o, pp, t0 in zip(outs, [p, p, q], [0.1, 0.3, 0.1]):
        assert rel_err(to_np(o), oracle_fine(M, 4.0, pp, u0, t0, dtau, 3)) <= KRYLOV_TOL


def test_payoff_kernel(bs):
    import torch
    from oracle import fd
    for p in PARAMS:
        M = 77
        g = bs.Grid(M, 4.0)
        u = torch.empty((M, M), device="cuda")
        bs.bs_payoff(g, p, u)
        torch.cuda.synchronize()
        X, Y = fd.mesh(M, 4.0)
        want = fd.payoff(p, X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64))
        assert np.max(np.abs(to_np(u) - want)) <= 1e-6
