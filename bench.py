"""Benchmark: Parareal time-to-tolerance vs serial fine stepping on one GB300.

One step = one Parareal solve (eq. parareal) to tol 1e-4 of the large single solve: a basket
call max(0.5 x + 0.5 y - 1, 0) on a 1024 x 1024 grid over [0,4]^2 (sigma1=0.3, sigma2=0.2,
rho=0.5, r=0.05, T=1), N=128 slices of 1024 implicit-Euler fine steps (FP32, temporally
blocked cluster tiles), FP64 defect norms, numerical coarse model with 4 steps per slice on
the 256 x 256 grid (bilinear restriction and prolongation).

  value   serial-fine-equivalent grid-point updates per second delivered by Parareal
          (M*M*N*fine_steps per solve / device time of the solve)
  e2e     the same through parareal_solve with host buffers: the initial state is copied
          from pinned host memory and the price surface u_N read back inside the timed region
  roofline      the fine stepper (the dominant kernel): algorithmic FP32 FLOP per second
                against the FP32 peak of the device's SMs at the measured maximum clock,
                with its DRAM bytes per launch from a committed ncu capture
                (profiles/traffic.json) while the kernel's sources are unchanged
  kernels       per-kernel event times, launches, rates and sweep counts
  exchange256   the 256 x 256 exchange-option workload (N=64 x 512 fine steps, rho in
                {-0.5, 0, 0.7}): time to tolerance, serial fine, coarse-sweep statistics
  coarse_models_128  the PINO network and the numerical G on 128 x 128 states, cost per state
                at one and at 128 states per call
  coarse_models_1024 G of one slice of the large solve: the PINO on its 256 x 256 grid
                (restricted and prolonged) against the numerical G on 256 x 256
  cpu_baseline  the FP64 oracle on one host core, a bounded sample of the large solve's
                serial fine stepping (one sparse LU factorisation, then implicit steps)
  clocks        nvidia-smi SM clock samples and throttle reasons during the timed region
  gpu_launches  the library's kernel launches inside the timed region (its own counters)
  serving       the serving sample: the first 200 requests of the seeded trace replayed through
                the server at 1.5x the one-at-a-time capacity (p50/p99 latency, solves/s
                against one request at a time)

Under torchrun with N ranks each GPU solves its own copy of the workload (replicas, weak
scaling; no data-path collective).  --slices instead partitions one solve's time slices over
the ranks (paper_2404_02521_gb300/slices.py; strong scaling).

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on a bounded sample
of the same workload, in the same unit.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "Parareal time-to-tol vs serial fine (1 GB300); fine pt-updates/s; p99 latency"
UNIT = "pt-updates/s"
L2_BYTES = 129 * 1024 * 1024


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def sm_count(dev_index=0):
    """Streaming multiprocessors of the device (queried, not assumed)."""
    import torch
    return int(torch.cuda.get_device_properties(dev_index).multi_processor_count)


# FP32 peak of an ALU-bound kernel: SMs x 128 FP32 lanes x 2 FLOP (FMA) x the maximum SM clock.
def fp32_peak_tflops(sm_mhz, sms):
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic FLOPs of one fine point-step with m Jacobi sweeps: each sweep is the 9-point
# update (5 FMA + 3 add + 1 multiply = 14 FLOP), plus b = dtau R_h w (16 FLOP), the
# compensated update (8 FLOP) and the next step's extrapolated guess (1 FMA = 2 FLOP) once
# per step.  A propagation of s steps takes m0 sweeps in its first (cold) step, m1 in the
# second (warm start), mx in steps 2-15 and mxl after them (extrapolated starts).
def fine_flops_per_point_step(m):
    return 14 * m + 26


EXTRAP_START, EXTRAP_LATE = 2, 16   # the library's default sweep schedule


def fine_flops_per_point_launch(m0, m1, mx, mxl, steps):
    f = 0
    for step in range(steps):
        m = m0 if step == 0 else m1 if step < EXTRAP_START else mx if step < EXTRAP_LATE else mxl
        f += fine_flops_per_point_step(m)
    return f


def fine_sweeps_total(m0, m1, mx, mxl, steps):
    t = 0
    for step in range(steps):
        t += m0 if step == 0 else m1 if step < EXTRAP_START else mx if step < EXTRAP_LATE else mxl
    return t


# Algorithmic FLOPs of one BiCGSTAB iteration per node of the coarse solve: two Jacobi-scaled
# 9-point products (15 FLOP each: 4 FMA, 2 multiplies, 3 adds), six dot-product terms (12) and
# the vector updates s, x, r, p (13).  Band variants with the degree-1 polynomial
# preconditioner M^{-1} = 2I - A^ evaluate two more scaled products and 2 y - A^ y twice (+34);
# with the degree-2 one, M^{-1} y = y + E(1.5 y + E y), four more products, w = 2.5 y - A^ y
# and (y + w) - A^ w twice (+68).
COARSE_FLOPS_PER_NODE_ITER = 55
COARSE_FLOPS_POLY_EXTRA = {0: 0, 1: 34, 2: 68}

# Algorithmic HBM bytes of the fine stepper per grid point and launch: the state read and
# written once in FP32 (8 B); a launch that blocks s steps moves 8 / s B per point-step.
FINE_ALG_BYTES_PER_POINT_LAUNCH = 8


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier_max(x, world):
    """Max of a per-rank value over all ranks (a tensor on the device the backend uses)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, t_max_ms):
    """Units per second of the whole job: every rank processed units_per_rank_step per step
    (weak scaling), and the job took the slowest rank's time."""
    return world * steps * units_per_rank_step / (t_max_ms / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


KERNEL_SOURCES = {
    "fine_ctile_kernel": ["paper_2404_02521_gb300/csrc/fine.cu", "paper_2404_02521_gb300/csrc/band.cuh",
                          "paper_2404_02521_gb300/csrc/common.cuh"],
    "fine_band_kernel": ["paper_2404_02521_gb300/csrc/fine.cu", "paper_2404_02521_gb300/csrc/band.cuh",
                         "paper_2404_02521_gb300/csrc/common.cuh"],
    "sweep_band_kernel": ["paper_2404_02521_gb300/csrc/coarse.cu", "paper_2404_02521_gb300/csrc/band.cuh",
                          "paper_2404_02521_gb300/csrc/common.cuh"],
}


def traffic_entry(kernel):
    """The committed ncu figures of a kernel (profiles/traffic.json), if its sources are
    unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kernel)
    if not ent:
        return None
    h = hashlib.sha256()
    for s in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    if ent.get("source_sha256") != h.hexdigest():
        return None
    return ent


def timed(stream, fn):
    """Device time of fn() in ms, CUDA events on the launching stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def large_arm(args, world, local):
    """The headline: Parareal on the 1024 x 1024 basket (numerical G on 256 x 256)."""
    import torch

    import paper_2404_02521_gb300 as bs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    pb = wl.large_cfg4()
    M, N = pb.M, pb.N
    g = bs.Grid(M, pb.xmax)
    g.set_coarse(256)
    U = torch.empty((N + 1, M, M), device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    bs.bs_set_option(bs.OPT_PHASE_TIMING, 1)

    def solve(flags=0):
        rc, k, d = bs.parareal_solve(g, pb.params, N, pb.fine_steps, bs.COARSE_NUM | flags, pb.coarse_steps,
                                     None, pb.tol, N, U, stream)
        return k, d

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    bs.bs_phase_stats(g)

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    total_ms, ks, defects = 0.0, [], None
    for _ in range(args.steps):
        flush.fill_(1.0)
        ms, (k, d) = timed(stream, solve)
        total_ms += ms
        ks.append(k)
        defects = d
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    phases = bs.bs_phase_stats(g)
    t_max_ms = barrier_max(total_ms, world)
    pts_per_step = M * M * N * pb.fine_steps
    value = whole_job_rate(pts_per_step, args.steps, world, t_max_ms)

    # serial fine stepping on the same GPU: the N slices one after another
    S = torch.empty((2, M, M), device=dev)
    sl = pb.params.T / N

    def serial():
        bs.bs_payoff(g, pb.params, S[0])
        for n in range(N):
            bs.fine_propagate_batched(g, [pb.params], [S[n % 2]], [S[(n + 1) % 2]], [n * sl], [pb.dtau_fine],
                                      pb.fine_steps, stream=stream)
    serial_ms, _ = timed(stream, serial)
    rel_diff = float((U[N] - S[N % 2]).abs().max() / S[N % 2].abs().max())
    bs.bs_phase_stats(g)

    # end to end through the C ABI with host buffers
    bs.bs_payoff(g, pb.params, U[0])
    torch.cuda.synchronize()
    u0_host = U[0].cpu().pin_memory()
    out_host = torch.empty((M, M), dtype=torch.float32).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U[0].copy_(u0_host, non_blocking=True)
        solve(bs.PARAREAL_USER_U0)
        out_host.copy_(U[N], non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
    e2e_value = whole_job_rate(pts_per_step, args.steps, world, barrier_max(e2e_ms, world))

    # roofline of the fine stepper from the event-timed F launches of the timed solves
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = sm_count(local)
    peak = fp32_peak_tflops(sm_max, sms)
    m0 = bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine, bs.START_COLD)
    m1 = bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine, bs.START_WARM)
    mx = bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine, bs.START_EXTRAP)
    mxl = bs.bs_fine_sweeps(g, pb.params, pb.dtau_fine, bs.START_EXTRAP_LATE)
    # state-propagations of F in the timed solves: iteration k covers slices k..N-1
    slices_f = sum(sum(N - kk for kk in range(k)) for k in ks)
    fine_flops = slices_f * M * M * fine_flops_per_point_launch(m0, m1, mx, mxl, pb.fine_steps)
    fine_s = phases["fine_ms"] / 1e3
    achieved = fine_flops / fine_s / 1e12 if fine_s > 0 else 0.0
    launches_f = max(1, phases["fine_launches"])
    ms_per_launch = phases["fine_ms"] / launches_f
    # Each F call splits its N - k states into chunks of at most 96 (one launch plan each), so
    # a launch carries on average the states of the timed F calls over their chunks.
    chunks = sum((N - kk + 95) // 96 for k in ks for kk in range(k))
    avg_states = slices_f / max(1, chunks)
    # DRAM bytes per launch: the committed capture's bytes per state and launch x avg_states
    ent = traffic_entry("fine_ctile_kernel")
    traffic = ent["dram_bytes_per_state_launch"] * avg_states if ent else None
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    alg_bytes_launch = avg_states * M * M * FINE_ALG_BYTES_PER_POINT_LAUNCH
    roof = {"kernel": "fine_ctile_kernel", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"FP32 lanes x 2 x {sm_max:.0f} MHz of {sms} SMs ({pk_kind} max clock)"}
    kernels = {
        "fine_ctile_kernel": {
            "ms_total": phases["fine_ms"], "launches": phases["fine_launches"], "ms_per_launch": ms_per_launch,
            "states_per_launch": avg_states, "bound": "alu", "achieved_tflops": achieved, "peak_tflops": peak,
            "frac": achieved / peak,
            "sweeps_per_step": {"cold": m0, "warm": m1, "extrapolated": mx, "extrapolated_after_16": mxl},
            "sweeps_per_slice": fine_sweeps_total(m0, m1, mx, mxl, pb.fine_steps),
            "hbm_algorithmic_gbs": alg_bytes_launch / (ms_per_launch / 1e3) / 1e9,
            "hbm_dram_gbs": (traffic / (ms_per_launch / 1e3) / 1e9) if traffic else None,
            "hbm_peak_gbs": hbm_peak,
        },
        "coarse_resampled": {"ms_total": phases["coarse_ms"], "launches": phases["coarse_launches"],
                             "note": "serial coarse sweep: restrict, BiCGSTAB on 256 x 256, prolong per slice"},
    }
    launches = phases["fine_launches"] + phases["coarse_launches"] + phases["other_launches"]
    del U, S
    return {
        "value": value, "t_ms": t_max_ms, "ks": ks, "defects": defects, "serial_ms": serial_ms,
        "rel_diff_vs_serial": rel_diff, "e2e": e2e_value, "roof": roof, "kernels": kernels, "clocks": clk,
        "launches": launches, "h2d": M * M * 4, "d2h": M * M * 4,
    }


def slices_arm(args, world, rank, local):
    """The large solve with its 128 time slices partitioned over the ranks (paper_2404_02521_gb300/
    slices.py: contiguous slices per GPU, u_n handed on point to point in the serial sweep, one
    FP64 all-reduce of the defect per iteration).  One solve per step for the whole job (strong
    scaling); the time is the slowest rank's."""
    import torch
    import torch.distributed as dist

    import paper_2404_02521_gb300 as bs
    from paper_2404_02521_gb300 import slices

    pb = wl.large_cfg4()
    g = bs.Grid(pb.M, pb.xmax)
    g.set_coarse(256)
    be = slices.GpuSlices(g, pb.params, pb.N, pb.fine_steps, pb.coarse_steps)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def solve():
        if rank == 0:
            be.initial()
        return slices.parareal_partitioned(be, pb.N, pb.tol, pb.N)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, ks = 0.0, []
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k, d = solve()
        torch.cuda.synchronize()
        total_ms += 1e3 * (time.perf_counter() - t0)
        ks.append(k)
    barrier(world)
    clk = clocks.stop()
    t_max = barrier_max(total_ms, world)
    pts = pb.M * pb.M * pb.N * pb.fine_steps
    value = args.steps * pts / (t_max / 1e3)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "basket1024_N128_fine1024_coarse4_on256", "grid": 1024, "slices": 128,
                   "fine_steps": 1024, "coarse_grid": 256, "tol": 1e-4,
                   "parallelism": f"time slices over {world} GPUs",
                   "slices_per_gpu": [b - a for a, b in slices.partition(pb.N, world)],
                   "l2": "flushed between timed steps (2x L2 buffer write); state 541 MB > L2"},
        "time_to_tol_ms_per_solve": t_max / args.steps, "parareal_iterations": ks[-1],
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 16 * (pb.N + 1)},
        "gpu_launches": None, "clocks": clk,
        "note": "host-timed (the driver synchronises on each iteration's defect); value and e2e are the same "
                "measurement: the initial state is formed on rank 0's GPU",
    }


def coarse_models(local):
    """The two coarse propagators on 128 x 128 basket states (the PINO workload's grid), per
    state, one state per call (the serial sweep) and 128 states per call
    (coarse_propagate_batched, as for concurrent solves): the PINO network (seeded random
    weights of the reading's architecture -- cost only) against the numerical G's 4 implicit
    steps."""
    import tempfile

    import torch

    import paper_2404_02521_gb300 as bs
    from paper_2404_02521_gb300 import pino_io

    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=3)
    fd_, path = tempfile.mkstemp(suffix=".bin")
    os.close(fd_)
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y, arch.layers,
                          arch.proj_hidden)
    net = bs.Pino(path)
    os.unlink(path)
    pb = wl.pino_cfg3()
    M = pb.M
    g = bs.Grid(M, pb.xmax)
    stream = torch.cuda.current_stream(torch.device("cuda", local))
    u0 = torch.empty((M, M), device="cuda")
    bs.bs_payoff(g, pb.params, u0)
    out = {}
    for B in (1, 128):
        ins = [u0.clone() for _ in range(B)]
        outs = [torch.empty_like(u0) for _ in range(B)]
        for name, kind, nt, steps in (("pino", bs.COARSE_PINO, net, 1), ("numerical_4_steps", bs.COARSE_NUM, None, 4)):
            def call():
                bs.coarse_propagate_batched(g, kind, nt, [pb.params] * B, ins, outs, [0.25] * B, pb.params.T / pb.N,
                                            steps, stream=stream)
            for _ in range(3):
                call()
            ms, _ = timed(stream, lambda: [call() for _ in range(5)])
            out[f"{name}_us_per_state_batch{B}"] = 1e3 * ms / 5 / B
    # the large solve's slice (1024 x 1024, dtau_slice = 1/128): the network on its 256 x 256
    # grid with restriction and prolongation, against the numerical G's 4 steps on 256 x 256
    pb4 = wl.large_cfg4()
    g4 = bs.Grid(pb4.M, pb4.xmax)
    u4 = torch.empty((pb4.M, pb4.M), device="cuda")
    o4 = torch.empty_like(u4)
    bs.bs_payoff(g4, pb4.params, u4)
    out4 = {}
    for name, kind, nt, steps, coarse in (("pino_net256", bs.COARSE_PINO, net, 1, 0),
                                          ("numerical_4_steps_on256", bs.COARSE_NUM, None, 4, 256)):
        g4.set_coarse(coarse)

        def call4():
            bs.coarse_propagate(g4, kind, nt, pb4.params, u4, o4, 0.25, pb4.params.T / pb4.N, steps,
                                stream=stream)
        for _ in range(3):
            call4()
        ms, _ = timed(stream, lambda: [call4() for _ in range(10)])
        out4[f"{name}_us_per_slice"] = 1e3 * ms / 10
    out4["note"] = ("G of one 1024 x 1024 slice of the large solve, as in its serial sweep; the PINO "
                    "row is cost only (seeded random weights)")
    return out, out4


def exchange_arm(args, local):
    """The 256 x 256 exchange-option workload (extra keys): Parareal to tol 1e-4 for each rho."""
    import torch

    import paper_2404_02521_gb300 as bs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    problems = [wl.exchange_cfg2(rho) for rho in wl.EXCHANGE_RHOS]
    pb0 = problems[0]
    M, N = pb0.M, pb0.N
    g = bs.Grid(M, pb0.xmax)
    U = torch.empty((N + 1, M, M), device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    bs.bs_set_option(bs.OPT_PHASE_TIMING, 1)

    def step():
        ks = []
        for pb in problems:
            rc, k, d = bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps,
                                         None, pb.tol, pb.N, U, stream)
            ks.append(k)
        return ks

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bs.bs_phase_stats(g)
    total_ms, ks = 0.0, []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ms, k = timed(stream, step)
        total_ms += ms
        ks.append(k)
    phases = bs.bs_phase_stats(g)
    krylov_iters = 0
    for pb in problems:   # one more (untimed) solve per rho: the solves are deterministic
        bs.parareal_solve(g, pb.params, pb.N, pb.fine_steps, bs.COARSE_NUM, pb.coarse_steps, None, pb.tol, pb.N,
                          U, stream)
        _, _, tot, ns = bs.bs_grid_stats(g, detail=True)
        krylov_iters += tot
    bs.bs_phase_stats(g)
    sl = pb0.params.T / N
    serial_ms = []
    for pb in problems:
        def serial():
            bs.bs_payoff(g, pb.params, U[0])
            for n in range(N):
                bs.fine_propagate_batched(g, [pb.params], [U[n]], [U[n + 1]], [n * sl], [pb.dtau_fine],
                                          pb.fine_steps, stream=stream)
        ms, _ = timed(stream, serial)
        serial_ms.append(ms)
    bs.bs_phase_stats(g)
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = sm_count(local)
    peak = fp32_peak_tflops(sm_max, sms)
    variant = bs.bs_coarse_variant(g, pb0.params, pb0.dtau_coarse)
    vinfo = bs.bs_coarse_variant_info(variant, M)
    flops_node_iter = COARSE_FLOPS_PER_NODE_ITER + COARSE_FLOPS_POLY_EXTRA[vinfo["poly"]]
    coarse_tflops = (args.steps * krylov_iters * M * M * flops_node_iter / (phases["coarse_ms"] / 1e3) / 1e12
                     if phases["coarse_ms"] > 0 else 0.0)
    per_solve = total_ms / (args.steps * len(problems))
    pts = sum(pb.M * pb.M * pb.N * pb.fine_steps for pb in problems)
    del U, flush
    return {
        "workload": "exchange256_N64_fine512_coarse4", "rho": list(wl.EXCHANGE_RHOS),
        "value": args.steps * pts / (total_ms / 1e3), "unit": UNIT,
        "time_to_tol_ms_per_solve": per_solve, "serial_fine_ms_per_solve": statistics.mean(serial_ms),
        "speedup_vs_serial_fine": statistics.mean(serial_ms) / per_solve, "parareal_iterations": ks[-1],
        "sweep_band_kernel": {
            "ms_total": phases["coarse_ms"], "launches": phases["coarse_launches"], "bound": "alu",
            "achieved_tflops": coarse_tflops, "peak_tflops": peak, "frac": coarse_tflops / peak,
            "band_variant": variant, "cluster_ctas": vinfo["ctas"], "polynomial_preconditioner_degree": vinfo["poly"],
            "quadratic_extrapolation": vinfo["quad"], "flops_per_node_iter": flops_node_iter,
            "krylov_iters_per_solve": krylov_iters / len(problems),
            "us_per_krylov_iter": 1e3 * phases["coarse_ms"] / max(1, args.steps * krylov_iters),
            "note": "serial coarse sweep on one thread-block cluster: latency-bound"},
        "fine_band_kernel": {"ms_total": phases["fine_ms"], "launches": phases["fine_launches"]},
    }


SERVE_COARSE_M = 256   # serving: grids above this run the numerical G on this coarse grid


def serving_run(args):
    """Serving sample: the first args.serve_requests requests of the seeded serving trace
    (seed 12345: basket/exchange 50/50, sigma ~ U[0.1,0.5], rho ~ U[-0.7,0.7],
    r ~ U[0,0.08], T ~ U[0.25,2], M in {64,128,256,512}, N in {16,32,64}; fine steps per slice
    64 doubled until the Jacobi bound is <= 0.7, one coarse step per slice, tol 1e-4; the
    numerical G on the request's grid, on 256 x 256 for the 512 x 512 requests as in the
    large solve).  Poisson arrivals at args.serve_load x the measured one-at-a-time capacity
    (above 1 the queue grows, so the solves/s show what batching and overlap add)."""
    import types

    import numpy as np
    import torch

    import paper_2404_02521_gb300 as bs
    from paper_2404_02521_gb300 import serving

    def with_coarse(r):
        f = {k.name: getattr(r, k.name) for k in dataclasses.fields(r)}
        return types.SimpleNamespace(**f, coarse_M=SERVE_COARSE_M if r.M > SERVE_COARSE_M else 0)

    n = args.serve_requests
    reqs = [with_coarse(t.problem) for t in wl.serving_trace(n, 0.0)]
    fs = [bs.bs_fine_steps_for(r.M, r.params, r.N) for r in reqs]
    # warm-up: one small request per grid size (autotuner, allocations, module loads)
    seen = {}
    for i, r in enumerate(reqs):
        seen.setdefault(r.M, i)
    warm = [with_coarse(wl.Problem("w", reqs[i].M, reqs[i].xmax, 16, 0, 1, dataclasses.replace(reqs[i].params, T=0.25)))
            for i in seen.values()]
    wfs = [bs.bs_fine_steps_for(r.M, r.params, r.N) for r in warm]
    serving.service_times(warm, wfs, [torch.empty((r.M, r.M), device="cuda") for r in warm])
    sv = bs.Server(16 << 30, 32)
    serving.replay(sv, warm, [0.0] * len(warm), [torch.empty((r.M, r.M), device="cuda") for r in warm])
    # one request at a time through parareal_solve, back to back
    alone = [torch.empty((r.M, r.M), device="cuda") for r in reqs]
    st = serving.service_times(reqs, fs, alone)
    svc = np.array([x["ms"] for x in st])
    capacity = n / (svc.sum() / 1e3)
    rate = args.serve_load * capacity
    rng = np.random.default_rng(12345 + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    arrivals -= arrivals[0]
    outs = [torch.empty((r.M, r.M), device="cuda") for r in reqs]
    res, makespan = serving.replay(sv, reqs, arrivals, outs)
    stats = sv.stats()
    sv.close()
    lat = np.array([r["latency_ms"] for r in res])
    fifo, fifo_span = serving.fifo_latencies(arrivals, svc)
    diff = max(float((a - b).abs().max() / b.abs().max()) for a, b in zip(outs, alone))
    return {
        "requests": n, "sample": f"first {n} requests of the seeded serving trace (seed 12345)",
        "coarse": f"numerical G on the request's grid, on {SERVE_COARSE_M}x{SERVE_COARSE_M} for larger grids",
        "grids": sorted({r.M for r in reqs}), "arrival_rate_per_s": rate,
        "load": args.serve_load, "one_at_a_time_capacity_per_s": capacity,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "solves_per_s": n / makespan, "makespan_s": makespan,
        "one_at_a_time": {"p50_ms": float(np.percentile(fifo, 50)), "p99_ms": float(np.percentile(fifo, 99)),
                          "solves_per_s": n / fifo_span, "service_ms_total": float(svc.sum())},
        "status_ok": sum(int(r["status"] == 0) for r in res),
        "parareal_iterations_mean": float(np.mean([r["iterations"] for r in res])),
        "results_max_rel_diff_vs_parareal_solve": diff,
        "fine_batches": stats["fine_batches"], "fine_slices_batched": stats["fine_items"],
        "slices_per_fine_batch": stats["fine_items"] / max(1, stats["fine_batches"]),
        "throughput_gain_vs_one_at_a_time": (n / makespan) / (n / fifo_span),
    }


_ORACLE_CACHE = {}


def oracle_sample(seconds_budget=15.0):
    """The FP64 oracle's serial fine stepping of the large solve: one sparse LU factorisation
    of the 1024 x 1024 implicit-Euler matrix (kept for later samples, as the oracle keeps it
    for every step of a solve), then as many implicit steps as fit the budget.  Returns the
    point-update rate of the steps, their count and time, and the factorisation time."""
    from oracle import fd
    pb = wl.large_cfg4()
    if "ie" not in _ORACLE_CACHE:
        t0 = time.perf_counter()
        _ORACLE_CACHE["ie"] = fd.ImplicitEuler(pb.M, pb.xmax, pb.params, pb.dtau_fine)
        _ORACLE_CACHE["factor_s"] = time.perf_counter() - t0
        _ORACLE_CACHE["u"] = fd.initial_state(pb.M, pb.xmax, pb.params)
        _ORACLE_CACHE["step"] = 0
    ie = _ORACLE_CACHE["ie"]
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds_budget:
        s = _ORACLE_CACHE["step"]
        _ORACLE_CACHE["u"] = ie.step(_ORACLE_CACHE["u"], (s + 1) * pb.dtau_fine)
        _ORACLE_CACHE["step"] = s + 1
        steps += 1
    dt = time.perf_counter() - t0
    return pb.M * pb.M * steps / dt, steps, dt, _ORACLE_CACHE["factor_s"]


def single_thread():
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(1)
    except Exception:
        return None


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ctx = single_thread()
    budget = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(budget / 4)
    vals, total_steps, total_s, factor_s = [], 0, 0.0, 0.0
    for _ in range(args.steps):
        v, st, dt, factor_s = oracle_sample(budget)
        vals.append(v)
        total_steps += st
        total_s += dt
    value = sum(vals) / len(vals)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "basket1024_N128_fine1024_coarse4_on256", "l2": "oracle runs on the CPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"FP64 sparse-LU serial fine stepping of the 1024x1024 basket "
                                   f"(dtau = 1/131072): {total_steps} implicit steps over {args.steps} "
                                   f"steps after one factorisation ({factor_s:.1f} s, not in the rate)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-exchange", action="store_true")
    ap.add_argument("--slices", action="store_true",
                    help="partition one large solve's time slices over the ranks (strong scaling) "
                         "instead of one independent solve per rank")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-load", type=float, default=1.5)
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    import paper_2404_02521_gb300 as bs
    bs.load()
    if args.slices:
        import torch.distributed as dist
        if not dist.is_initialized():   # the driver's collectives need a group, even of one
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29531")
            dist.init_process_group("nccl", rank=rank, world_size=world)
        out = slices_arm(args, world, rank, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        dist.destroy_process_group()
        return
    r = large_arm(args, world, local)
    ex = exchange_arm(args, local) if (not args.no_exchange and world == 1) else None
    cm, cm4 = coarse_models(local) if (not args.no_exchange and world == 1) else (None, None)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        ctx = single_thread()
        v, st, dt, factor_s = oracle_sample(15.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 sparse-LU serial fine stepping of the 1024x1024 basket (dtau = 1/131072): "
                         f"{st} of 131072 implicit steps in {dt:.1f} s after one factorisation "
                         f"({factor_s:.1f} s, not in the rate)"}
    serving_res = None
    if not args.no_serving and world == 1:
        serving_res = serving_run(args)
    per_solve = r["t_ms"] / args.steps
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_solve, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "basket1024_N128_fine1024_coarse4_on256",
                   "grid": 1024, "slices": 128, "fine_steps": 1024, "coarse_steps": 4, "coarse_grid": 256,
                   "coarse": "numerical (BiCGSTAB) on 256x256 with bilinear resampling", "tol": 1e-4,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "flushed between timed steps (2x L2 buffer write); state 541 MB > L2"},
        "time_to_tol_ms_per_solve": per_solve,
        "serial_fine_ms_per_solve": r["serial_ms"],
        "speedup_vs_serial_fine": r["serial_ms"] / per_solve,
        "parareal_iterations": r["ks"][-1],
        "defects": r["defects"],
        "rel_diff_vs_serial_fine": r["rel_diff_vs_serial"],
        "roofline": r["roof"],
        "kernels": r["kernels"],
        "exchange256": ex,
        "coarse_models_128": cm,
        "coarse_models_1024": cm4,
        "cpu_baseline": cpu,
        "e2e": {"value": r["e2e"], "unit": UNIT, "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "serving": serving_res,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
