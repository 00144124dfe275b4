"""Helpers shared by the GPU tests: run the CUDA path through the C ABI binding and the
FP64 oracle on the same float32 inputs."""
import numpy as np

import workloads as wl
from oracle import fd

FP32_FINE_TOL = 1e-5     # max|V_gpu - V_oracle| <= 1e-5 * max|V| for FP32 fine stepping


def dtau_for(M, p, q_target=0.4):
    """A step size whose Jacobi contraction on an M-grid is about q_target."""
    s2 = max(p.sigma1, p.sigma2) ** 2
    return q_target / (s2 * (M - 2) ** 2 * (1.0 + abs(p.rho)))


def to_gpu(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def to_np(t):
    return t.detach().cpu().double().numpy()


def oracle_fine(M, xmax, p, u0_f32, tau0, dtau, nsteps):
    ie = fd.ImplicitEuler(M, xmax, p, dtau)
    return ie.propagate(np.asarray(u0_f32, dtype=np.float64), tau0, nsteps)


def rel_err(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def start_state(M, xmax, p, kind, seed=0):
    X, Y = fd.mesh(M, xmax)
    if kind == "payoff":
        u = fd.payoff(p, X, Y)
    else:
        rng = np.random.default_rng(seed)
        u = np.abs(wl.random_field(rng, M)) + fd.payoff(p, X, Y)
        g = fd.dirichlet(p)(X, Y, 0.1)
        u[M - 1, :] = g[M - 1, :]
        u[:, M - 1] = g[:, M - 1]
    return u.astype(np.float32)
