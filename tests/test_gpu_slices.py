"""parareal_sweep_range, the serial coarse sweep over a range of slices that drivers use to
partition the slices over GPUs (paper_2404_02521_gb300/slices.py): on one GPU, sweeps over
consecutive ranges compose to the whole sweep -- bit for bit with G on a coarse grid (every
slice's coarse solve starts afresh), and to the Krylov tolerance with G on the state grid (the
cluster sweep's coarse solves extrapolate their first guess from the previous slice's
increments, a history that restarts at a range boundary) -- and the partitioned driver with
one rank reproduces parareal_solve bit for bit."""
import os
import socket

import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


def _fine(bs, g, pb, U, Fb, lo, hi):
    sl = pb.params.T / pb.N
    n = range(lo, hi)
    bs.fine_propagate_batched(g, [pb.params] * len(n), [U[i] for i in n], [Fb[i] for i in n],
                              [i * sl for i in n], [pb.dtau_fine] * len(n), pb.fine_steps)


@pytest.mark.parametrize("M,Mc", [(64, 0), (128, 64)])
def test_range_sweeps_compose(bs, M, Mc):
    import torch
    pb = wl.Problem("range", M, 4.0, 8, 64 if M == 64 else 256, 2, wl.exchange_cfg2(0.7).params)
    g = bs.Grid(pb.M, pb.xmax)
    if Mc:
        g.set_coarse(Mc)
    arrays = []
    for cuts in ([0, pb.N], [0, 3, 5, pb.N]):
        U = torch.zeros((pb.N + 1, M, M), device="cuda")
        Fb = torch.zeros((pb.N, M, M), device="cuda")
        Gold = torch.zeros_like(Fb)
        nrm = torch.zeros(2 * (pb.N + 1), dtype=torch.float64, device="cuda")
        bs.bs_payoff(g, pb.params, U[0])
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            bs.parareal_sweep_range(g, pb.params, pb.N, pb.coarse_steps, -1, lo, hi, U, None, Gold, nrm)
        for k in range(2):
            _fine(bs, g, pb, U, Fb, k, pb.N)
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                if hi > k:
                    bs.parareal_sweep_range(g, pb.params, pb.N, pb.coarse_steps, k, max(lo, k), hi, U, Fb,
                                            Gold, nrm)
        torch.cuda.synchronize()
        arrays.append((U, Gold, nrm))
    if Mc:
        assert torch.equal(arrays[0][0], arrays[1][0])
        assert torch.equal(arrays[0][1], arrays[1][1])
        assert torch.equal(arrays[0][2][2:], arrays[1][2][2:])
    else:   # three times the coarse propagator's parity bound, as for the two Parareal drivers
        U0, U1 = arrays[0][0], arrays[1][0]
        assert float((U0 - U1).abs().max() / U0.abs().max()) <= 6e-5
    # two iterations of the phase-by-phase driver give the whole sweeps' iterate
    U2 = torch.empty_like(arrays[0][0])
    try:
        bs.bs_set_option(bs.OPT_PIPELINE, 0)
        bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps, None, 0.0, 2, U2)
        torch.cuda.synchronize()
    finally:
        bs.bs_set_option(bs.OPT_PIPELINE, 1)
    assert torch.equal(U2, arrays[0][0])


def test_range_sweep_rejects_bad_ranges(bs):
    import torch
    pb = wl.Problem("range", 32, 4.0, 4, 32, 1, wl.basket_cfg1().params)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.zeros((pb.N + 1, pb.M, pb.M), device="cuda")
    Fb = torch.zeros((pb.N, pb.M, pb.M), device="cuda")
    nrm = torch.zeros(2 * (pb.N + 1), dtype=torch.float64, device="cuda")
    for k, lo, hi in ((-2, 0, 4), (1, 0, 4), (0, 2, 2), (0, 0, 5), (4, 4, 4)):
        with pytest.raises(bs.BSError):
            bs.parareal_sweep_range(g, pb.params, pb.N, 1, k, lo, hi, U, Fb, Fb, nrm)


def test_partitioned_driver_one_rank_matches_parareal_solve(bs):
    # the driver of slices.py with a single rank (a gloo group of one: no hand-off) on the GPU
    # backend: the iteration count, defects and iterate of parareal_solve's phase-by-phase
    # driver, bit for bit
    import torch
    import torch.distributed as dist
    from paper_2404_02521_gb300 import slices
    pb = wl.Problem("part", 64, 4.0, 8, 64, 4, wl.basket_cfg1().params)
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        g = bs.Grid(pb.M, pb.xmax)

        class CpuReduce(slices.GpuSlices):   # gloo reduces host tensors
            def max_tensor(self, values):
                return torch.tensor(values, dtype=torch.float64)

        be = CpuReduce(g, pb.params, pb.N, pb.fine_steps, pb.coarse_steps)
        be.initial()
        k, defects = slices.parareal_partitioned(be, pb.N, 1e-4, pb.N)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    U = torch.empty_like(be.U)
    try:
        bs.bs_set_option(bs.OPT_PIPELINE, 0)
        rc, k0, d0 = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps, None,
                                       1e-4, pb.N, U)
        torch.cuda.synchronize()
    finally:
        bs.bs_set_option(bs.OPT_PIPELINE, 1)
    assert k == k0 and defects == d0
    assert torch.equal(be.U, U)
