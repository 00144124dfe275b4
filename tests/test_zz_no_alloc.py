"""parareal_solve_noalloc: the Parareal entry point for callers that may not allocate device
memory (a latency-critical pricing path, or a host framework that owns all device memory).
Its scratch is a fixed device array inside the library, shared by every call, so this test
makes two calls in a row and checks each against parareal_solve, which allocates its own
workspace.  The file is named so that pytest collects it last."""
import ctypes as C
import os
import subprocess
import sys

import pytest

import workloads as wl
from tests.gpu_util import FP32_FINE_TOL, rel_err, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


def test_noalloc_matches_parareal_solve_on_two_calls(bs):
    import torch
    problems = [wl.Problem("basket64", 64, 4.0, 8, 64, 4, wl.basket_cfg1().params),
                wl.Problem("exchange64", 64, 4.0, 8, 64, 4, wl.exchange_cfg2(0.7).params)]
    for pb in problems:
        g = bs.Grid(pb.M, pb.xmax)
        ref = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
        try:   # the no-allocation entry point runs F and the sweep as alternating phases
            bs.bs_set_option(bs.OPT_PIPELINE, 0)
            rc0, k0, d0 = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM,
                                            pb.coarse_steps, None, pb.tol, pb.N, ref)
            torch.cuda.synchronize()
        finally:
            bs.bs_set_option(bs.OPT_PIPELINE, 1)
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            before = bs.bs_device_allocations()
            rc, k, d = bs.parareal_solve_noalloc(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps,
                                                 pb.coarse_steps, pb.tol, pb.N, out)
            torch.cuda.synchronize()
            assert bs.bs_device_allocations() == before   # the call allocated nothing
            assert rc == rc0 == 0 and k == k0
            assert rel_err(to_np(out), to_np(ref)) <= FP32_FINE_TOL
            assert all(abs(a - b) <= 1e-12 + 1e-9 * abs(b) for a, b in zip(d, d0))


# A fresh process whose first call is the no-allocation entry point: no band variant has been
# measured for M there, so the coarse sweep runs the default variant without tuning (tuning
# would allocate).  Its result is compared with parareal_solve's (which then tunes M): the
# coarse solves of two variants agree to the Krylov tolerance, not bitwise, so the iterates are
# held to three times the coarse propagator's parity bound of 2e-5 max|V| and the defects to
# 1e-3 relative, as for the two Parareal drivers.
_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import torch
import paper_2404_02521_gb300 as bs
import workloads as wl
from tests.gpu_util import rel_err, to_np
bs.load()
pb = wl.Problem("exchange128", 128, 4.0, 16, 256, 4, wl.exchange_cfg2(-0.5).params)   # Jacobi bound 0.52
out = torch.full(((pb.N + 1), pb.M, pb.M), float("nan"), device="cuda")
before = bs.bs_device_allocations()
rc, k, d = bs.parareal_solve_noalloc(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps,
                                     pb.coarse_steps, pb.tol, pb.N, out)
torch.cuda.synchronize()
assert bs.bs_device_allocations() == before, "the first call allocated"
g = bs.Grid(pb.M, pb.xmax)
ref = torch.empty_like(out)
bs.bs_set_option(bs.OPT_PIPELINE, 0)
rc0, k0, d0 = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM,
                                pb.coarse_steps, None, pb.tol, pb.N, ref)
torch.cuda.synchronize()
err = rel_err(to_np(out), to_np(ref))
print("FRESH", rc, k, k0, err)
assert rc == rc0 == 0 and k == k0 and err <= 6e-5, (rc, rc0, k, k0, err)
assert all(abs(a - b) <= 1e-3 * b + 1e-6 for a, b in zip(d, d0)), (d, d0)
"""


def test_noalloc_first_call_in_a_fresh_process():
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FRESH" in r.stdout


def test_noalloc_rejects_sizes_beyond_capacity(bs):
    import torch
    u = torch.empty(1, device="cuda")
    p = bs.to_params(wl.exchange_cfg2(0.7).params)
    k = C.c_int(0)
    rc = bs.load().parareal_solve_noalloc(512, 4.0, C.byref(p), 64, 512, 4, 1e-4, 64,
                                          u.data_ptr(), C.byref(k), None, None)
    assert rc == -1
    assert "exceeds the fixed scratch capacity" in bs.last_error()
    # within the node capacity, but beyond the grids that fit one cluster
    rc = bs.load().parareal_solve_noalloc(512, 4.0, C.byref(p), 16, 512, 4, 1e-4, 16,
                                          u.data_ptr(), C.byref(k), None, None)
    assert rc == -1
    assert "M <= 256" in bs.last_error()
