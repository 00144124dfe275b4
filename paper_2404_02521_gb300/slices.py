"""Parareal with its time slices partitioned over the ranks of a process group (one GPU per
rank): the space-time layout of Sec. 4.3 reduced to its time axis, since one GB300 holds a whole
state.

Rank r owns the contiguous slices [a_r, b_r) (balanced, `partition`).  One iteration k of
eq. (parareal):

  1. F on the rank's open slices max(a_r, k) .. b_r - 1, all at once (no communication);
  2. the serial coarse sweep: rank r receives u_{a_r}^{k+1} from rank r - 1 (point to point),
     sweeps its slices -- G, the correction F + (G_new - G_old) and the slice norms in one
     library call -- and sends u_{b_r}^{k+1} to rank r + 1.  A rank whose slices are all
     exact (b_r <= k) neither sweeps nor sends, and its successor does not wait;
  3. the defect of reading c5 from one FP64 max all-reduce of each rank's largest squared
     norms, delta = sqrt(max ||du||^2) / sqrt(max ||u||^2).

The all-reduce is started asynchronously and, from the second iteration on while the defect is
above 10 tol, F of the next iteration is enqueued before its result is known (it only reads
the rank's own, already corrected states), so a rank that has finished its part of the sweep
does not idle while later ranks sweep; the defect is read back through its own event, not
behind that F.  The arithmetic is the
single-GPU driver's: every result equals parareal_solve's phase-by-phase iteration
(BS_OPT_PIPELINE = 0) on one GPU.

The driver is written against a small backend interface, so that the same code runs on GPUs
through the library (`GpuSlices`) and, in the tests, on CPU ranks with any other propagator.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def partition(N: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous slice ranges [a_r, b_r) of N slices over `world` ranks, sizes differing by at
    most one (the first N % world ranks get the extra slice)."""
    if N < 1 or world < 1:
        raise ValueError(f"partition: N={N} world={world}")
    base, extra = divmod(N, world)
    out, a = [], 0
    for r in range(world):
        b = a + base + (1 if r < extra else 0)
        out.append((a, b))
        a = b
    return out


def defect_from(num2: float, den2: float) -> float:
    """Reading c5 from the largest squared norms."""
    import math
    return math.sqrt(num2) / math.sqrt(den2) if den2 > 0.0 else math.sqrt(num2)


class SliceBackend:
    """What the driver needs from a rank's propagators and storage (full-size arrays indexed by
    the global slice number; only the rank's own entries are used)."""

    def fine(self, n_lo: int, n_hi: int) -> None:
        """F of slices [n_lo, n_hi): Fb[n] = F(U[n])."""
        raise NotImplementedError

    def sweep(self, k: int, n_lo: int, n_hi: int) -> None:
        """The serial sweep over [n_lo, n_hi) (k = -1: the initial sweep)."""
        raise NotImplementedError

    def state(self, n: int):
        """U[n] as a tensor the process group can send and receive into."""
        raise NotImplementedError

    def norms(self, n_lo: int, n_hi: int) -> Sequence[Tuple[float, float]]:
        """(||U[n]||^2, ||dU[n]||^2) for n in (n_lo, n_hi] (written by the last sweeps)."""
        raise NotImplementedError

    def max_tensor(self, values: Sequence[float]):
        """A float64 tensor of `values` on the device the process group reduces on."""
        raise NotImplementedError

    def read_async(self, t):
        """Start copying the reduced tensor t to the host; returns a callable that waits for
        the copy alone (not for work enqueued after it) and returns the values."""
        vals = t.double().cpu().tolist()
        return lambda: vals


def parareal_partitioned(backend: SliceBackend, N: int, tol: float, Kmax: int, group=None):
    """Run Parareal with this rank's share of the slices.  Returns (k_done, defects); the rank's
    states U[a_r + 1 .. b_r] hold the last iterate (rank 0 also U[0]).  k_done = N or a defect
    <= tol means converged, as for parareal_solve."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if N < world:
        raise ValueError(f"parareal_partitioned: N={N} slices for {world} ranks (at least one each)")
    a, b = partition(N, world)[rank]
    prev, nxt = rank - 1, rank + 1

    def gsrc(r):
        return dist.get_global_rank(group, r) if group is not None else r

    # the initial coarse sweep, rank after rank
    if rank > 0:
        dist.recv(backend.state(a), src=gsrc(prev), group=group)
    backend.sweep(-1, a, b)
    if rank < world - 1:
        dist.send(backend.state(b), dst=gsrc(nxt), group=group)
    own_u = [nu for nu, _ in backend.norms(a, b)]   # ||U_n||^2, n = a+1 .. b
    den2 = max(own_u)

    defects: List[float] = []
    k = 0
    f_done = False
    while k < Kmax:
        lo = max(a, k)
        if not f_done and lo < b:
            backend.fine(lo, b)
        if lo < b:
            if rank > 0 and a > k:
                dist.recv(backend.state(a), src=gsrc(prev), group=group)
            backend.sweep(k, lo, b)
            if rank < world - 1:
                dist.send(backend.state(b), dst=gsrc(nxt), group=group)
        # largest squared norms of the rank's slices: ||du|| over the slices this sweep moved
        # (n > k), ||u|| over all of the rank's slices (those below k keep their last value)
        num2 = 0.0
        if lo < b:
            nrm = backend.norms(lo, b)
            num2 = max(du for _, du in nrm)
            own_u[lo - a:] = [nu for nu, _ in nrm]   # the rank's slices below lo keep theirs
            den2 = max(own_u)
        t = backend.max_tensor([num2, den2])
        work = dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group, async_op=True)
        work.wait()   # orders the result before later work on the rank's stream
        result = backend.read_async(t)
        # F of the next iteration while later ranks still sweep and the reduction is in flight
        # -- from the second iteration on, and unless the last defect was already within
        # 10 tol (then this iteration is likely the last, and the speculative F would only
        # delay what follows the solve)
        f_done = False
        if k >= 1 and defects[-1] > 10.0 * tol and k + 1 < Kmax and max(a, k + 1) < b:
            backend.fine(max(a, k + 1), b)
            f_done = True
        vals = result()
        delta = defect_from(vals[0], vals[1])
        defects.append(delta)
        k += 1
        if delta <= tol:
            break
    return k, defects


class GpuSlices(SliceBackend):
    """The rank's GPU through the library: F by fine_propagate_batched, the sweep by
    parareal_sweep_range, states in full-size device arrays on the current device."""

    def __init__(self, grid, params, N: int, fine_steps: int, coarse_steps: int, device=None):
        import torch

        from . import _lib
        self.lib = _lib
        self.g, self.p, self.N = grid, params, N
        self.fine_steps, self.coarse_steps = fine_steps, coarse_steps
        M = grid.M
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.U = torch.zeros((N + 1, M, M), dtype=torch.float32, device=dev)
        self.Fb = torch.zeros((N, M, M), dtype=torch.float32, device=dev)
        self.Gold = torch.zeros((N, M, M), dtype=torch.float32, device=dev)
        self.nrm = torch.zeros(2 * (N + 1), dtype=torch.float64, device=dev)
        self.dev = dev
        self.slice = params.T / N

    def initial(self):
        self.lib.bs_payoff(self.g, self.p, self.U[0])

    def fine(self, n_lo, n_hi):
        n = range(n_lo, n_hi)
        self.lib.fine_propagate_batched(self.g, [self.p] * len(n), [self.U[i] for i in n], [self.Fb[i] for i in n],
                                        [i * self.slice for i in n], [self.slice / self.fine_steps] * len(n),
                                        self.fine_steps)

    def sweep(self, k, n_lo, n_hi):
        self.lib.parareal_sweep_range(self.g, self.p, self.N, self.coarse_steps, k, n_lo, n_hi, self.U,
                                      None if k < 0 else self.Fb, self.Gold, self.nrm)

    def state(self, n):
        return self.U[n]

    def norms(self, n_lo, n_hi):
        h = self.nrm[2 * (n_lo + 1): 2 * (n_hi + 1)].cpu().tolist()
        return [(h[2 * i], h[2 * i + 1]) for i in range(n_hi - n_lo)]

    def max_tensor(self, values):
        import torch
        return torch.tensor(values, dtype=torch.float64, device=self.dev)

    def read_async(self, t):
        import torch
        host = torch.empty(t.numel(), dtype=torch.float64, pin_memory=True)
        host.copy_(t, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record()

        def wait():
            ev.synchronize()
            return host.tolist()
        return wait
