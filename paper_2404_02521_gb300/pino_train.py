"""Offline training of the PINO coarse propagator (Sec. 3.5) -- tooling, not the hot path.

Training data are slice pairs (u(tau_n), u(tau_n + dtau)) produced by this library's own
fine propagator on the GPU: random sigma1, sigma2 ~ U[0.1, 0.5], rho ~ U[-0.7, 0.7],
r ~ U[0, 0.08], basket and exchange payoffs, on an M x M grid of [0, 4]^2 with N slices of
fine_steps implicit steps (the states along each trajectory are the "initial conditions
sampled at different time steps" of Sec. 3.5).  The network (same architecture the CUDA
library evaluates: lifting, L Fourier layers with modes_x x 2*modes_y retained modes,
pointwise layers, ReLU, projection) predicts the increment u(tau_n + dtau) - u(tau_n).

Loss (Sec. 3.5, eq. bs_totalloss, adapted to a slice map): mean squared error against the
fine solution, plus a physics term -- the residual of eq. (bse_change_variable) of the
prediction at the collocation points, discretised by eq. (fd) with the slice as one implicit
step -- and a boundary term on the far edges.  The physics term and its gradient are the
library's kernel (pino_physics_loss); the network's forward and backward passes are PyTorch.
Adam, learning rate 1e-3 decayed by 0.96 at fixed intervals.

Usage (on a GPU machine):
    python -m paper_2404_02521_gb300.pino_train --out weights.bin [--problems 256] [--iters 6000] [--slices 12,64]
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from paper_2404_02521_gb300 import _lib as bs  # noqa: E402
from paper_2404_02521_gb300 import pino_io  # noqa: E402


class FNO(torch.nn.Module):
    def __init__(self, cin=9, width=32, mx=12, my=12, layers=4, hidden=128):
        super().__init__()
        self.mx, self.my, self.width = mx, my, width
        self.lift = torch.nn.Linear(cin, width)
        scale = 1.0 / (width * width)
        self.spec = torch.nn.ParameterList([
            torch.nn.Parameter(scale * torch.randn(2 * my, mx, width, width, dtype=torch.cfloat))
            for _ in range(layers)])
        self.pw = torch.nn.ModuleList([torch.nn.Linear(width, width) for _ in range(layers)])
        self.p1 = torch.nn.Linear(width, hidden)
        self.p2 = torch.nn.Linear(hidden, 1)

    def spectral(self, v, R):
        # v [B][C][M][M]; keep ky in [0, my) U [M - my, M), kx in [0, mx)
        B, C, M, _ = v.shape
        V = torch.fft.rfft2(v)
        out = torch.zeros(B, C, M, M // 2 + 1, dtype=torch.cfloat, device=v.device)
        my, mx = self.my, self.mx
        out[:, :, :my, :mx] = torch.einsum("bcyx,yxco->boyx", V[:, :, :my, :mx], R[:my])
        out[:, :, M - my:, :mx] = torch.einsum("bcyx,yxco->boyx", V[:, :, M - my:, :mx], R[my:])
        return torch.fft.irfft2(out, s=(M, M))

    def forward(self, a):
        # a [B][9][M][M] -> increment [B][M][M]
        v = self.lift(a.permute(0, 2, 3, 1)).permute(0, 3, 1, 2)
        for R, pw in zip(self.spec, self.pw):
            k = self.spectral(v, R)
            p = pw(v.permute(0, 2, 3, 1)).permute(0, 3, 1, 2)
            v = torch.relu(k + p)
        h = torch.relu(self.p1(v.permute(0, 2, 3, 1)))
        return self.p2(h)[..., 0]

    def export(self, path):
        w = {
            "lift_w": self.lift.weight.detach().T.cpu().double().numpy(),
            "lift_b": self.lift.bias.detach().cpu().double().numpy(),
            "spec_w": np.stack([R.detach().cpu().numpy().astype(np.complex128) for R in self.spec]),
            "pw_w": np.stack([p.weight.detach().T.cpu().double().numpy() for p in self.pw]),
            "pw_b": np.stack([p.bias.detach().cpu().double().numpy() for p in self.pw]),
            "proj1_w": self.p1.weight.detach().T.cpu().double().numpy(),
            "proj1_b": self.p1.bias.detach().cpu().double().numpy(),
            "proj2_w": self.p2.weight.detach()[0].cpu().double().numpy(),
            "proj2_b": float(self.p2.bias.detach().cpu()[0]),
        }
        pino_io.write_weights(path, w, 9, self.width, self.mx, self.my, len(self.spec),
                              self.p1.out_features)


class PhysicsLoss(torch.autograd.Function):
    """Per-sample PDE term of the loss, eq. bs_totalloss's MSE_f, on the device: the mean
    square of the residual of eq. (bse_change_variable) over the collocation points, from
    the library (forward and gradient in one kernel launch)."""

    @staticmethod
    def forward(ctx, pred, u_prev, params, dtau, grid):
        pred = pred.detach().contiguous()
        u_prev = u_prev.detach().contiguous()
        B = pred.shape[0]
        loss = torch.empty(B, dtype=torch.float64, device=pred.device)
        grad = torch.empty_like(pred)
        bs.pino_physics_loss(grid, params, list(pred), list(u_prev), [dtau] * B, loss, list(grad))
        ctx.save_for_backward(grad)
        return loss.to(pred.dtype)

    @staticmethod
    def backward(ctx, g_loss):
        (grad,) = ctx.saved_tensors
        return g_loss.view(-1, 1, 1) * grad, None, None, None, None


def sample_params(prm):
    """bs_params of the samples of a batch (the residual needs sigma1, sigma2, rho, r only)."""
    return [wl.Params(float(a), float(b), float(c), float(d)) for a, b, c, d in prm.tolist()]


def generate(M, N, fine_steps, n_problems, seed, device, rough=0.0):
    """Trajectories u_0..u_N of random problems from the library's fine propagator."""
    rng = np.random.default_rng(seed)
    g = bs.Grid(M, 4.0)
    params = []
    for k in range(n_problems):
        payoff = wl.BASKET if k % 2 == 0 else wl.EXCHANGE
        params.append(wl.random_params(rng, payoff, 1.0))
    U = torch.empty((n_problems, N + 1, M, M), device=device)
    for k, p in enumerate(params):
        bs.bs_payoff(g, p, U[k, 0])
    sl = 1.0 / N
    for n in range(N):
        # one batched launch per slice over all problems (chunks of 96 inside the library)
        bs.fine_propagate_batched(g, params, [U[k, n] for k in range(n_problems)],
                                  [U[k, n + 1] for k in range(n_problems)], [n * sl] * n_problems,
                                  [sl / fine_steps] * n_problems, fine_steps)
    torch.cuda.synchronize()
    prm = torch.tensor([[p.sigma1, p.sigma2, p.rho, p.r] for p in params], device=device,
                       dtype=torch.float32)
    # Perturbed states: Parareal applies G to iterates that are not on the fine trajectory, so
    # the network must also learn F's response near it.  Each state gets a smooth random
    # perturbation (a few low Fourier modes, relative size up to 5%, zero on the far edges)
    # and is propagated over one slice by the fine solver.
    gen = torch.Generator(device="cpu").manual_seed(seed + 1)
    x = torch.linspace(0.0, 1.0, M, device=device)
    mask = ((1.0 - x).view(1, M) * (1.0 - x).view(M, 1))
    edge = torch.ones(M, M, device=device)
    edge[-1, :] = 0.0
    edge[:, -1] = 0.0
    P0 = torch.empty((n_problems, N, M, M), device=device)
    P1 = torch.empty_like(P0)
    for k in range(n_problems):
        coef = torch.randn(N, 4, 4, generator=gen).to(device)
        amp = 0.05 * torch.rand(N, 1, 1, generator=gen).to(device)
        modes = torch.stack([torch.sin(math.pi * (a + 1) * x) for a in range(4)])   # [4][M]
        eta = torch.einsum("nab,ay,bx->nyx", coef, modes, modes) * mask / 4.0
        if rough > 0.0:
            # Rough perturbations as well (every other slice): white noise, which the fine
            # propagator damps within a slice.  Parareal's coarse propagator must damp it too:
            # a network that passes high-frequency error through unchanged (G ~ I beyond its
            # retained modes) lets it accumulate along the slices instead of correcting it.
            noise = torch.randn(N, M, M, generator=gen).to(device) * edge
            odd = (torch.arange(N, device=device) % 2 == 1).view(N, 1, 1)
            eta = torch.where(odd, rough * noise / 0.05, eta)
        scale = U[k, :N].abs().amax(dim=(1, 2)).view(N, 1, 1)
        P0[k] = U[k, :N] + amp * scale * eta
    for n in range(N):
        bs.fine_propagate_batched(g, params, [P0[k, n] for k in range(n_problems)],
                                  [P1[k, n] for k in range(n_problems)], [n * sl] * n_problems,
                                  [sl / fine_steps] * n_problems, fine_steps)
    torch.cuda.synchronize()
    return U, prm, P0, P1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--M", type=int, default=128)
    ap.add_argument("--slices", default="12,64", help="slice counts N of [0, 1] to train on")
    ap.add_argument("--fine-dtau", type=float, default=1.0 / 32768)
    ap.add_argument("--problems", type=int, default=256, help="trajectories per slice count")
    ap.add_argument("--iters", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--physics-weight", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--rough", type=float, default=0.0,
                    help="relative size of the white-noise perturbations (0: smooth ones only)")
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args()
    dev = torch.device("cuda")
    torch.manual_seed(args.seed)
    bs.load()
    t0 = time.time()
    M = args.M
    sets = []
    for q, N in enumerate(int(v) for v in args.slices.split(",")):
        fine = max(1, int(round(1.0 / (N * args.fine_dtau))))
        U, prm, P0, P1 = generate(M, N, fine, args.problems, args.seed + 7 * q, dev, args.rough)
        sets.append(dict(N=N, U=U, prm=prm, P0=P0, P1=P1, dtau=1.0 / N))
        print(f"data: {args.problems} trajectories x {N} slices of {fine} fine steps "
              f"({time.time() - t0:.1f} s)", flush=True)
    h = 4.0 / (M - 1)
    grid = bs.Grid(M, 4.0)
    x = torch.arange(M, device=dev, dtype=torch.float32) * h
    Xg, Yg = x.view(1, M).expand(M, M), x.view(M, 1).expand(M, M)
    model = FNO().to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=args.lr)
    sched = torch.optim.lr_scheduler.StepLR(opt, step_size=max(1, args.iters // 100), gamma=0.96)
    n_train = int(0.9 * args.problems)
    gen = torch.Generator(device="cpu").manual_seed(args.seed)

    def batch(ds, lo, hi, B):
        N, U, P0, P1, dtau = ds["N"], ds["U"], ds["P0"], ds["P1"], ds["dtau"]
        k = torch.randint(lo, hi, (B,), generator=gen)
        n = torch.randint(0, N, (B,), generator=gen)
        pert = torch.rand(B, generator=gen) < 0.5     # half on-trajectory, half perturbed
        kd, nd, pd = k.to(dev), n.to(dev), pert.to(dev).view(B, 1, 1)
        u0 = torch.where(pd, P0[kd, nd], U[kd, nd])
        u1 = torch.where(pd, P1[kd, nd], U[kd, nd + 1])
        p = ds["prm"][kd]
        one = torch.ones(B, M, M, device=dev)
        tau = (nd.float() * dtau).view(B, 1, 1)
        a = torch.stack([u0, Xg.expand(B, M, M), Yg.expand(B, M, M), tau * one, dtau * one,
                         p[:, 0].view(B, 1, 1) * one, p[:, 1].view(B, 1, 1) * one,
                         p[:, 2].view(B, 1, 1) * one, p[:, 3].view(B, 1, 1) * one], dim=1)
        return a, u0, u1, p, dtau

    for it in range(args.iters):
        a, u0, u1, p, dtau = batch(sets[it % len(sets)], 0, n_train, args.batch)
        pred = u0 + model(a)
        # squared error relative to each sample's own increment: late slices, whose increments
        # are small, weigh as much as the early ones near the payoff kink
        inc2 = torch.mean((u1[:, :-1, :-1] - u0[:, :-1, :-1]) ** 2, dim=(1, 2)) + 1e-12
        data = torch.mean(torch.mean((pred[:, :-1, :-1] - u1[:, :-1, :-1]) ** 2, dim=(1, 2)) / inc2) * 1e-4
        bnd = torch.mean((pred[:, -1, :] - u1[:, -1, :]) ** 2) + torch.mean((pred[:, :, -1] - u1[:, :, -1]) ** 2)
        phys = torch.mean(PhysicsLoss.apply(pred, u0, sample_params(p), dtau, grid)) * dtau ** 2
        loss = data + 0.1 * bnd + args.physics_weight * phys
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if it % 1000 == 0 or it == args.iters - 1:
            msg = []
            with torch.no_grad():
                for ds in sets:
                    a, u0, u1, p, _ = batch(ds, n_train, args.problems, 64)
                    pred = u0 + model(a)
                    rel = torch.sqrt(torch.mean((pred - u1) ** 2) / torch.mean((u1 - u0) ** 2))
                    msg.append(f"N={ds['N']}: {rel.item():.3f}")
            print(f"it {it} loss {loss.item():.3e} held-out increment rel. rms err " + ", ".join(msg),
                  flush=True)
    model.export(args.out)
    print(f"wrote {args.out} after {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main()
