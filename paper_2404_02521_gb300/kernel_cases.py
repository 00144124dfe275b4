"""Single-kernel workloads for profiling the library's kernels (e.g. under ncu).

    python -m paper_2404_02521_gb300.kernel_cases <case> [--reps R]

Each case builds its inputs on the device, runs the kernel once untimed and then R times,
and prints the CUDA-event time per launch.  The cases are the launches of the benchmark
workloads, one kernel each:

  fine256    F on all 64 slices of the 256x256 exchange workload, 512 steps (one launch)
  coarse256  the initial serial coarse sweep of that workload (64 slices x 4 BiCGSTAB steps)
  tile1024   F on 48 slices of a 1024x1024 basket grid, 40 steps of the large-solve step size
             (temporally blocked cluster tiles; 48 x 4 MB of state exceeds the 129 MB L2).  The
             launch plan of one call: the cold first step split over two launches, the warm
             second step with the third, two extrapolated steps per launch up to step 14, then
             four steps of five sweeps per launch (the twelfth launch, steps 23-26, is the
             steady state of the large solve)
  solve256   one Parareal solve of that workload (rho = 0.7): payoff, initial coarse sweep,
             then per iteration the batched F launch and a correcting coarse sweep
  coarse512  coarse propagation of one 512x512 state, 4 steps (global-memory BiCGSTAB)
  large1024  the large single solve: basket on 1024x1024, N = 128 slices of 1024 fine steps,
             numerical G with 4 steps per slice on a 256x256 grid (bilinear resampling);
             prints Parareal time to tolerance, iterations and serial fine stepping time
  pino128    the PINO coarse propagator on 64 states of 128x128 (random weights)
  pino128b   the PINO on 128 states of 128x128 in one coarse_propagate_batched call (random
             weights): the network's GEMM chain with the states as extra rows or blocks
  resample1024  Parareal to K = N = 4 on 1024x1024 basket states with numerical G on the 256x256
             grid (bilinear restriction and prolongation kernels, 64 fine steps per slice)
  fine3_64   three-asset F: 16 states of 64^3 nodes, 64 implicit steps (19-point stencil)
  coarse3_64 three-asset G: one 64^3 basket state, 4 BiCGSTAB-solved steps of 0.025
"""
from __future__ import annotations

import argparse
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _timed(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def case_fine256(bs, wl, torch):
    pb = wl.exchange_cfg2(0.7)
    M, N = pb.M, pb.N
    g = bs.Grid(M, pb.xmax)
    U = torch.empty((N, M, M), device="cuda")
    bs.bs_payoff(g, pb.params, U[0])
    U[1:].copy_(U[0].expand(N - 1, M, M))
    F = torch.empty_like(U)
    sl = pb.params.T / N
    args = ([pb.params] * N, list(U), list(F), [n * sl for n in range(N)], [pb.dtau_fine] * N,
            pb.fine_steps)
    return lambda: bs.fine_propagate_batched(g, *args)


def case_coarse256(bs, wl, torch):
    pb = wl.exchange_cfg2(0.7)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    bs.bs_coarse_variant(g, pb.params, pb.dtau_coarse)

    def run():
        # Kmax = 0: the payoff and the initial coarse sweep only
        try:
            bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                              None, pb.tol, 0, U)
        except bs.BSError:
            pass   # "tol not met after 0 iterations" is the expected status
    return run


def case_solve256(bs, wl, torch):
    pb = wl.exchange_cfg2(0.7)
    g = bs.Grid(pb.M, pb.xmax)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    return lambda: bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM,
                                     pb.coarse_steps, None, pb.tol, pb.N, U)


def case_tile1024(bs, wl, torch):
    p = wl.basket_cfg1().params
    M, B, steps = 1024, 48, 40
    g = bs.Grid(M, 4.0)
    U = torch.empty((B, M, M), device="cuda")
    bs.bs_payoff(g, p, U[0])
    U[1:].copy_(U[0].expand(B - 1, M, M))
    F = torch.empty_like(U)
    dtau = p.T / (128 * 1024)
    args = ([p] * B, list(U), list(F), [0.01 * n for n in range(B)], [dtau] * B, steps)
    return lambda: bs.fine_propagate_batched(g, *args)


def case_coarse512(bs, wl, torch):
    p = wl.Params(0.25, 0.35, 0.7, 0.03, payoff=wl.EXCHANGE)
    M = 512
    g = bs.Grid(M, 4.0)
    u = torch.empty((M, M), device="cuda")
    bs.bs_payoff(g, p, u)
    o = torch.empty_like(u)
    return lambda: bs.coarse_propagate(g, bs.COARSE_NUM, None, p, u, o, 0.25, 4.0 / 256, 4)


def case_pino128(bs, wl, torch):
    from paper_2404_02521_gb300 import pino_io
    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=3)
    fd, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd)
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y,
                          arch.layers, arch.proj_hidden)
    net = bs.Pino(path)
    os.unlink(path)
    pb = wl.pino_cfg3()
    M, N = pb.M, pb.N
    g = bs.Grid(M, pb.xmax)
    U = torch.empty((N + 1, M, M), device="cuda")

    def run():
        try:
            bs.parareal_solve(g, pb.params, N, pb.fine_steps, bs.COARSE_PINO, 1, net, pb.tol, 0, U)
        except bs.BSError:
            pass   # Kmax = 0: payoff and the initial PINO sweep only
    run.net = net
    return run


def case_pino128b(bs, wl, torch):
    from paper_2404_02521_gb300 import pino_io
    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=3)
    fd, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd)
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y,
                          arch.layers, arch.proj_hidden)
    net = bs.Pino(path)
    os.unlink(path)
    pb = wl.pino_cfg3()
    g = bs.Grid(pb.M, pb.xmax)
    u0 = torch.empty((pb.M, pb.M), device="cuda")
    bs.bs_payoff(g, pb.params, u0)
    ins = [u0.clone() for _ in range(128)]
    outs = [torch.empty_like(u0) for _ in range(128)]

    def run():
        bs.coarse_propagate_batched(g, bs.COARSE_PINO, net, [pb.params] * 128, ins, outs, [0.25] * 128,
                                    pb.params.T / pb.N)
    run.net = net
    return run


def case_large1024(bs, wl, torch):
    import time
    pb = wl.large_cfg4()
    g = bs.Grid(pb.M, pb.xmax)
    g.set_coarse(256)
    U = torch.empty((pb.N + 1, pb.M, pb.M), device="cuda")
    state = {}

    def run():
        t0 = time.perf_counter()
        rc, k, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                     None, pb.tol, pb.N, U)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        state["solve"] = (rc, k, d, 1e3 * (t1 - t0))
        if "serial" not in state:   # serial fine stepping once: N launches of one slice
            S = torch.empty_like(U)
            bs.bs_payoff(g, pb.params, S[0])
            sl = pb.params.T / pb.N
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for n in range(pb.N):
                bs.fine_propagate_batched(g, [pb.params], [S[n]], [S[n + 1]], [n * sl], [pb.dtau_fine],
                                          pb.fine_steps)
            torch.cuda.synchronize()
            state["serial"] = 1e3 * (time.perf_counter() - t0)
            state["err"] = float((U - S).abs().max() / S.abs().max())
        rc, k, d, ms = state["solve"]
        print(f"large1024: rc={rc} k={k} defects={['%.1e' % x for x in d]} parareal={ms:.0f} ms "
              f"serial_fine={state['serial']:.0f} ms rel_diff_vs_serial={state['err']:.1e}", flush=True)
    return run


def case_resample1024(bs, wl, torch):
    # the large solve's coarse model at reduced length: 1024^2 basket states, numerical G on
    # the 256^2 grid (restriction, coarse solve, prolongation with the correction and the
    # defect norms), N = 4 slices of 64 fine steps at the large solve's fine step size
    import dataclasses
    base = wl.large_cfg4()
    T = 4 * 64 * base.dtau_fine
    p = dataclasses.replace(base.params, T=T)
    M, N = base.M, 4
    g = bs.Grid(M, base.xmax)
    g.set_coarse(256)
    U = torch.empty((N + 1, M, M), device="cuda")
    return lambda: bs.parareal_solve(g, p, N, 64, bs.COARSE_NUM, base.coarse_steps, None, 0.0, N, U)


def case_fine3_64(bs, wl, torch):
    # three assets: 16 states of 64^3 nodes (a 3-asset basket), 64 implicit steps each
    import types
    p = types.SimpleNamespace(sigma=(0.3, 0.2, 0.25), rho=(0.5, -0.3, 0.2), r=0.05, strike=1.0,
                              w=(0.4, 0.35, 0.25), payoff=wl.BASKET)
    M, B, steps, dtau = 64, 16, 64, 1.0 / 4096
    U = torch.empty((B, M, M, M), device="cuda")
    bs.bs_payoff3(M, 4.0, p, U[0])
    U[1:].copy_(U[0].expand(B - 1, M, M, M))
    F = torch.empty_like(U)
    return lambda: bs.fine_propagate3(M, 4.0, p, list(U), list(F), [0.01 * b for b in range(B)], dtau, steps)


def case_coarse3_64(bs, wl, torch):
    # three assets: G over one slice of 0.1 (4 implicit steps) on one 64^3 basket state
    import types
    p = types.SimpleNamespace(sigma=(0.3, 0.2, 0.25), rho=(0.5, -0.3, 0.2), r=0.05, strike=1.0,
                              w=(0.4, 0.35, 0.25), payoff=wl.BASKET)
    M = 64
    u = torch.empty((M, M, M), device="cuda")
    bs.bs_payoff3(M, 4.0, p, u)
    out = torch.empty_like(u)
    return lambda: bs.coarse_propagate3(M, 4.0, p, u, out, 0.0, 0.1, 4)


CASES = {"fine256": case_fine256, "coarse256": case_coarse256, "solve256": case_solve256,
         "pino128b": case_pino128b,
         "tile1024": case_tile1024,
         "coarse512": case_coarse512, "pino128": case_pino128, "large1024": case_large1024,
         "resample1024": case_resample1024, "fine3_64": case_fine3_64,
         "coarse3_64": case_coarse3_64}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--coarse-variant", type=int, default=-1,
                    help="force this coarse band variant (skips the autotuner's timing launches)")
    args = ap.parse_args()
    import torch

    import paper_2404_02521_gb300 as bs
    import workloads as wl
    bs.load()
    bs.bs_set_option(bs.OPT_COARSE_VARIANT, args.coarse_variant)
    fn = CASES[args.case](bs, wl, torch)
    ms = _timed(fn, args.reps)
    print(f"{args.case}: " + " ".join(f"{t:.3f}" for t in ms) + " ms per launch group")


if __name__ == "__main__":
    main()
