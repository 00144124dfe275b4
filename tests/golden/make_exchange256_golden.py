"""Write tests/golden/exchange256_rho*.json: FP64 oracle serial fine solution of the
256x256 exchange-option workload (sigma1=0.25, sigma2=0.35, r=0.03, T=1, N=64 slices of
512 implicit-Euler steps), sampled at fixed nodes after selected slices.

Calls only oracle/ (and the seeded workload description).  Run from the repository root:
    python tests/golden/make_exchange256_golden.py            # all three rho values
    python tests/golden/make_exchange256_golden.py 0.7        # one value
Takes about 12 minutes per rho on one CPU core.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import fd  # noqa: E402

SLICES = (1, 2, 8, 32, 64)


def sample_nodes(M, seed=2024, n_random=384):
    rng = np.random.default_rng(seed)
    j = rng.integers(0, M, n_random)
    i = rng.integers(0, M, n_random)
    diag = np.arange(0, M, 8)
    j = np.concatenate([j, diag, np.full(16, M // 2), np.full(16, M - 2)])
    i = np.concatenate([i, diag, np.arange(16) * (M // 16), np.arange(16) * (M // 16)])
    return j.astype(int), i.astype(int)


def run(rho):
    pb = wl.exchange_cfg2(rho)
    t0 = time.time()
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
    u = fd.initial_state(pb.M, pb.xmax, pb.params)
    j, i = sample_nodes(pb.M)
    out = {"workload": pb.name, "M": pb.M, "xmax": pb.xmax, "N": pb.N,
           "fine_steps": pb.fine_steps, "params": pb.params.__dict__, "rows": j.tolist(),
           "cols": i.tolist(), "slices": {}, "maxabs": {}}
    for n in range(pb.N):
        u = F(u, n)
        if (n + 1) in SLICES:
            out["slices"][str(n + 1)] = u[j, i].tolist()
            out["maxabs"][str(n + 1)] = float(np.max(np.abs(u)))
    out["oracle_seconds"] = time.time() - t0
    path = os.path.join(HERE, f"exchange256_rho{rho:+.1f}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    return path


if __name__ == "__main__":
    rhos = [float(a) for a in sys.argv[1:]] or list(wl.EXCHANGE_RHOS)
    for rho in rhos:
        print(run(rho), flush=True)
