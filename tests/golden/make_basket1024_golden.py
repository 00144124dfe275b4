"""Write tests/golden/basket1024_slice0.json: the FP64 oracle's fine propagation of the first
slice of the large single solve -- the basket call max(0.5 x + 0.5 y - 1, 0) on a 1024x1024
grid over [0,4]^2 (sigma1=0.3, sigma2=0.2, rho=0.5, r=0.05, T=1, N=128 slices of 1024
implicit-Euler steps, dtau = 1/131072) from the payoff -- sampled at fixed nodes after steps
16, 128 and 1024 (eq. fd with implicit Euler, Sec. 3.2; reading c4 for the step size).

Calls only oracle/ (and the seeded workload description).  Run from the repository root:
    python tests/golden/make_basket1024_golden.py
Takes about ten minutes on one CPU core (one sparse LU factorisation of the 1024^2 system,
then 1024 triangular solves).
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

CHECKPOINTS = (16, 128, 1024)


def sample_nodes(M, seed=1024, n_random=512):
    rng = np.random.default_rng(seed)
    j = rng.integers(0, M, n_random)
    i = rng.integers(0, M, n_random)
    # the payoff's kink x + y = 2 (i + j = (M - 1) / 2), the far edges' neighbours and a diagonal
    k = np.arange(0, M // 2, 8)
    kink_j, kink_i = k, (M - 1) // 2 - k
    diag = np.arange(0, M, 16)
    j = np.concatenate([j, kink_j, diag, np.full(32, M - 2), np.arange(32) * (M // 32)])
    i = np.concatenate([i, kink_i, diag, np.arange(32) * (M // 32), np.full(32, M - 2)])
    return j.astype(int), i.astype(int)


def run():
    pb = wl.large_cfg4()
    t0 = time.time()
    ie = fd.ImplicitEuler(pb.M, pb.xmax, pb.params, pb.dtau_fine)
    u = fd.initial_state(pb.M, pb.xmax, pb.params)
    j, i = sample_nodes(pb.M)
    out = {"workload": pb.name, "M": pb.M, "xmax": pb.xmax, "N": pb.N, "fine_steps": pb.fine_steps,
           "dtau": pb.dtau_fine, "tau0": 0.0, "params": pb.params.__dict__, "rows": j.tolist(),
           "cols": i.tolist(), "steps": {}, "maxabs": {}}
    for s in range(pb.fine_steps):
        u = ie.step(u, (s + 1) * pb.dtau_fine)
        if (s + 1) in CHECKPOINTS:
            out["steps"][str(s + 1)] = u[j, i].tolist()
            out["maxabs"][str(s + 1)] = float(np.max(np.abs(u)))
    out["oracle_seconds"] = time.time() - t0
    path = os.path.join(HERE, "basket1024_slice0.json")
    with open(path, "w") as f:
        json.dump(out, f)
    return path


if __name__ == "__main__":
    print(run(), flush=True)
