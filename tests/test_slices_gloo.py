"""Parareal with the time slices partitioned over ranks (paper_2404_02521_gb300/slices.py: the
time axis of the paper's space-time layout, Sec. 4.3, eq. parareal): CPU ranks on the gloo
backend run the driver with the FP64 oracle's F and G, and every rank's slices, the iteration
count and the defects must equal the single-process textbook Parareal of oracle/parareal.py.
This covers the partition, the point-to-point hand-off of u_n in the serial sweep, the skipped
exact slices and the all-reduced defect."""
import os
import socket

import numpy as np
import pytest

import workloads as wl
from paper_2404_02521_gb300.slices import SliceBackend, parareal_partitioned, partition


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class OracleSlices(SliceBackend):
    """A rank's propagators on CPU: the oracle's F and G (FP64), full-size states."""

    def __init__(self, pb):
        import torch
        from oracle import fd
        self.F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
        self.G = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.coarse_steps)
        self.U = torch.zeros((pb.N + 1, pb.M, pb.M), dtype=torch.float64)
        self.U[0] = torch.from_numpy(fd.initial_state(pb.M, pb.xmax, pb.params))
        self.Fb = np.zeros((pb.N, pb.M, pb.M))
        self.Gold = np.zeros((pb.N, pb.M, pb.M))
        self.nrm = np.zeros(2 * (pb.N + 1))
        self.fine_calls = []

    def fine(self, n_lo, n_hi):
        self.fine_calls.append((n_lo, n_hi))
        for n in range(n_lo, n_hi):
            self.Fb[n] = self.F(self.U[n].numpy(), n)

    def sweep(self, k, n_lo, n_hi):
        for n in range(n_lo, n_hi):
            u = self.U[n].numpy()
            if k < 0:
                new = self.G(u, n)
                self.Gold[n] = new
            else:
                g = self.Gold[n] if n == k else self.G(u, n)   # u_k is exact after k iterations
                new = self.Fb[n] + (g - self.Gold[n])
                self.Gold[n] = g
            old = self.U[n + 1].numpy().copy()
            self.U[n + 1] = __import__("torch").from_numpy(new)
            self.nrm[2 * (n + 1)] = float(np.sum(new * new))
            self.nrm[2 * (n + 1) + 1] = float(np.sum((new - old) ** 2)) if k >= 0 else 0.0

    def state(self, n):
        return self.U[n]

    def norms(self, n_lo, n_hi):
        return [(self.nrm[2 * n], self.nrm[2 * n + 1]) for n in range(n_lo + 1, n_hi + 1)]

    def max_tensor(self, values):
        import torch
        return torch.tensor(values, dtype=torch.float64)


def _worker(rank, world, port, pb, tol, Kmax, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    be = OracleSlices(pb)
    k, defects = parareal_partitioned(be, pb.N, tol, Kmax)
    a, b = partition(pb.N, world)[rank]
    out[rank] = (k, defects, a, b, be.U[a + 1: b + 1].numpy().copy(), be.fine_calls)
    dist.barrier()
    dist.destroy_process_group()


def run_ranks(world, pb, tol, Kmax):
    import torch.multiprocessing as mp
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), pb, tol, Kmax, out), nprocs=world, join=True)
        return dict(out)


def oracle_parareal(pb, tol, Kmax):
    from oracle import fd
    from oracle import parareal as opr
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
    G = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.coarse_steps)
    u0 = fd.initial_state(pb.M, pb.xmax, pb.params)
    return opr.parareal(u0, F, G, pb.N, tol, Kmax)


def test_partition_is_contiguous_and_balanced():
    for N in (1, 5, 8, 64, 128):
        for world in range(1, min(N, 9) + 1):
            parts = partition(N, world)
            assert parts[0][0] == 0 and parts[-1][1] == N
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world,N,tol,Kmax", [(2, 6, 1e-6, 6), (2, 6, 0.0, 3), (3, 7, 1e-6, 7)])
def test_partitioned_parareal_equals_single_process(world, N, tol, Kmax):
    pb = wl.Problem("slices", 14, 4.0, N, 12, 1, wl.exchange_cfg2(0.7).params)
    res = run_ranks(world, pb, tol, Kmax)
    Uo, ko, do, _ = oracle_parareal(pb, tol, Kmax)
    for rank in range(world):
        k, defects, a, b, U, fine_calls = res[rank]
        assert k == ko
        assert np.allclose(defects, do, rtol=1e-12, atol=0.0)
        # the rank's slices are the single-process iterate bit for bit
        assert np.array_equal(U, Uo[a + 1: b + 1]), rank
        # F ran only on open slices (never on the exact prefix of a later iteration)
        assert all(lo >= a and hi == b for lo, hi in fine_calls)
    if tol == 0.0:
        assert ko == Kmax
