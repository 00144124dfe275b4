"""Write tests/golden/cash_or_nothing301.json: FP64 oracle serial fine solution of the paper's
own problem (Sec. 3.2): a two-asset cash-or-nothing call on [0,300]^2 with dx = dy = 1
(301 x 301 nodes), S1 = S2 = 100, c = 1, r = 1, sigma1 = sigma2 = 0.3, rho = 0.5, T = 1,
N = 10 slices (coarse step 0.1, Sec. 4.1).  Fine steps per slice: 3 (the paper's three
substeps), doubled until the Gershgorin bound of a fine step is <= 0.7 (reading: the fine
propagator solves each step by Jacobi sweeps).  Sampled nodes after slices 1, 2, 5 and 10,
and the error of the final state against the closed form (eq. solution).

A second file, cash_or_nothing301_paper_steps.json, holds the paper's own step sizes: three
fine substeps per slice and one coarse step (Sec. 4.1), together with the oracle's Parareal
iterations and defects to tol 1e-4 with that numerical coarse model.

Calls only oracle/ (and the seeded workload description).  Run from the repository root:
    python tests/golden/make_paper_golden.py            # both files
    python tests/golden/make_paper_golden.py paper      # the paper-steps file only (~1 min)
Takes about ten minutes on one CPU core.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import closed_forms as cf  # noqa: E402
from oracle import fd  # noqa: E402
from oracle import parareal as opr  # noqa: E402

SLICES = (1, 2, 5, 10)


def fine_steps(pb, qmax=0.7, start=3):
    s = start
    while fd.jacobi_contraction(pb.M, pb.xmax, pb.params, pb.params.T / pb.N / s) > qmax:
        s *= 2
    return s


def sample_nodes(M, seed=301):
    rng = np.random.default_rng(seed)
    j = rng.integers(0, M, 320)
    i = rng.integers(0, M, 320)
    # the region around the strikes, where the price varies fastest
    g = np.arange(60, 181, 8)
    jj, ii = np.meshgrid(g, g, indexing="ij")
    return np.concatenate([j, jj.ravel()]).astype(int), np.concatenate([i, ii.ravel()]).astype(int)


def main(fs=None, name="cash_or_nothing301.json", parareal=False):
    pb0 = wl.paper_cash_or_nothing(N=10)
    fs = fine_steps(pb0) if fs is None else fs
    pb = wl.paper_cash_or_nothing(N=10, fine_steps=fs)
    t0 = time.time()
    F = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, pb.fine_steps)
    u = fd.initial_state(pb.M, pb.xmax, pb.params)
    j, i = sample_nodes(pb.M)
    out = {"workload": pb.name, "M": pb.M, "xmax": pb.xmax, "N": pb.N, "fine_steps": fs,
           "coarse_steps": 1, "params": pb.params.__dict__, "rows": j.tolist(), "cols": i.tolist(),
           "slices": {}, "maxabs": {}}
    for n in range(pb.N):
        u = F(u, n)
        if (n + 1) in SLICES:
            out["slices"][str(n + 1)] = u[j, i].tolist()
            out["maxabs"][str(n + 1)] = float(np.max(np.abs(u)))
    X, Y = fd.mesh(pb.M, pb.xmax)
    p = pb.params
    exact = cf.cash_or_nothing(X, Y, p.strike, p.strike2, p.cash, p.r, p.sigma1, p.sigma2, p.rho, p.T)
    out["closed_form_rel_l2"] = float(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    out["closed_form_rel_max"] = float(np.max(np.abs(u - exact)) / np.max(np.abs(exact)))
    if parareal:
        G = fd.SlicePropagator(pb.M, pb.xmax, pb.params, pb.N, 1)
        u0 = fd.initial_state(pb.M, pb.xmax, pb.params)
        U, k, defects, hist = opr.parareal(u0, F, G, pb.N, 1e-4, pb.N)
        out["parareal_k"] = int(k)
        out["parareal_defects"] = [float(x) for x in defects]
        out["parareal_final"] = U[pb.N][j, i].tolist()
        out["coarse_closed_form_rel_l2"] = float(np.linalg.norm(hist[0][pb.N] - exact) / np.linalg.norm(exact))
    out["oracle_seconds"] = time.time() - t0
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["closed_form_rel_l2"], out["closed_form_rel_max"], out["oracle_seconds"])


if __name__ == "__main__":
    if len(sys.argv) < 2 or sys.argv[1] != "paper":
        main()
    main(fs=3, name="cash_or_nothing301_paper_steps.json", parareal=True)
