"""GPU parity of the PINO training loss's PDE term (Sec. 3.5, eq. bs_totalloss) and its
gradient against the FP64 oracle on the same float32 inputs."""
import numpy as np
import pytest

import workloads as wl
from oracle import fd, physics
from tests.gpu_util import to_gpu, to_np

pytestmark = pytest.mark.gpu

# The residual is formed in FP32 from O(1) values: about 16 rounded operations per point, and
# the difference (u_pred - u_prev) - dtau R_h u_pred cancels by up to two decimal digits on
# these fields, so each residual carries a relative error of about 16 * 6e-8 * 100 ~ 1e-4 at
# worst; the loss and the gradient (nine residuals per node) inherit that bound.
PHYS_REL_TOL = 1e-4


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


PARAMS = [wl.Params(0.3, 0.2, 0.5, 0.05, payoff=wl.BASKET),
          wl.Params(0.25, 0.35, -0.6, 0.03, payoff=wl.EXCHANGE),
          wl.Params(0.45, 0.15, 0.0, 0.08, payoff=wl.BASKET)]


@pytest.mark.parametrize("M", [33, 64, 130])
def test_physics_loss_and_gradient_match_oracle(bs, M):
    import torch
    rng = np.random.default_rng(M)
    g = bs.Grid(M, 4.0)
    X, Y = fd.mesh(M, 4.0)
    dtaus = [1.0 / 64, 1.0 / 12, 0.002]
    prev, pred = [], []
    for p, dt in zip(PARAMS, dtaus):
        u0 = fd.payoff(p, X, Y) + 0.1 * wl.random_field(rng, M)
        u1 = u0 + dt * wl.random_field(rng, M, scale=0.5)
        prev.append(np.asarray(u0, dtype=np.float32))
        pred.append(np.asarray(u1, dtype=np.float32))
    tp = [to_gpu(a) for a in pred]
    tv = [to_gpu(a) for a in prev]
    loss = torch.empty(len(PARAMS), dtype=torch.float64, device="cuda")
    grads = [torch.empty((M, M), device="cuda") for _ in PARAMS]
    bs.pino_physics_loss(g, PARAMS, tp, tv, dtaus, loss, grads)
    torch.cuda.synchronize()
    got = loss.cpu().numpy()
    for b, (p, dt) in enumerate(zip(PARAMS, dtaus)):
        w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
        u1 = pred[b].astype(np.float64)
        u0 = prev[b].astype(np.float64)
        want = physics.loss(u1, u0, dt, w)
        assert abs(got[b] - want) <= PHYS_REL_TOL * want, (b, got[b], want)
        gw = physics.loss_grad(u1, u0, dt, w)
        gg = to_np(grads[b])
        assert np.max(np.abs(gg - gw)) <= PHYS_REL_TOL * np.max(np.abs(gw)), b
    # the loss alone (no gradient) gives the same values
    loss2 = torch.empty_like(loss)
    bs.pino_physics_loss(g, PARAMS, tp, tv, dtaus, loss2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(loss2.cpu().numpy(), got, rtol=1e-12)


def test_physics_loss_of_a_fine_step_is_small(bs):
    # a slice predicted by the library's own fine propagator with one implicit step of the
    # slice length satisfies the discretised PDE up to the FP32 solve: its loss is far below
    # that of a perturbed prediction
    import torch
    M, p = 64, PARAMS[0]
    g = bs.Grid(M, 4.0)
    X, Y = fd.mesh(M, 4.0)
    dt = 1e-4
    u0 = to_gpu(fd.payoff(p, X, Y))
    u1 = torch.empty_like(u0)
    bs.fine_propagate_batched(g, [p], [u0], [u1], [0.0], [dt], 1)
    bad = u1 + 1e-3 * to_gpu(wl.random_field(np.random.default_rng(1), M))
    loss = torch.empty(2, dtype=torch.float64, device="cuda")
    bs.pino_physics_loss(g, [p, p], [u1, bad], [u0, u0], [dt, dt], loss)
    torch.cuda.synchronize()
    good, worse = loss.cpu().numpy()
    assert good <= 1e-6 * worse


def test_physics_loss_rejects_bad_arguments(bs):
    import torch
    M = 16
    g = bs.Grid(M, 4.0)
    u = torch.zeros((M, M), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(bs.BSError):
        bs.pino_physics_loss(g, [PARAMS[0]], [u], [u], [0.0], loss)
    with pytest.raises(bs.BSError):
        bs.pino_physics_loss(g, [PARAMS[0]], [u], [u], [0.01], loss, [u])   # grad aliases u_pred


def test_trainer_backpropagates_the_physics_term(bs):
    # the training loop's autograd wrapper returns the kernel's loss and gradient
    import torch
    from paper_2404_02521_gb300 import pino_train
    M, dt = 48, 1.0 / 32
    rng = np.random.default_rng(5)
    g = bs.Grid(M, 4.0)
    X, Y = fd.mesh(M, 4.0)
    prev = np.stack([fd.payoff(p, X, Y) for p in PARAMS[:2]]).astype(np.float32)
    pred = (prev + dt * np.stack([wl.random_field(rng, M) for _ in range(2)])).astype(np.float32)
    prm = torch.tensor([[p.sigma1, p.sigma2, p.rho, p.r] for p in PARAMS[:2]], device="cuda")
    t_pred = torch.tensor(pred, device="cuda", requires_grad=True)
    t_prev = torch.tensor(prev, device="cuda")
    out = pino_train.PhysicsLoss.apply(t_pred, t_prev, pino_train.sample_params(prm), dt, g)
    (out * torch.tensor([1.0, 3.0], device="cuda")).sum().backward()
    for b, wgt in enumerate([1.0, 3.0]):
        p = PARAMS[b]
        w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
        want_l = physics.loss(pred[b].astype(np.float64), prev[b].astype(np.float64), dt, w)
        assert abs(float(out[b].detach()) - want_l) <= PHYS_REL_TOL * want_l
        want_g = wgt * physics.loss_grad(pred[b].astype(np.float64), prev[b].astype(np.float64), dt, w)
        got_g = t_pred.grad[b].detach().cpu().double().numpy()
        assert np.max(np.abs(got_g - want_g)) <= PHYS_REL_TOL * np.max(np.abs(want_g))


def test_pino_training_runs_end_to_end(bs, tmp_path):
    # a few iterations of the trainer (data from the library's F, the physics term from the
    # library's kernel): it finishes, and the network it writes loads and runs as G
    import re
    import subprocess
    import sys

    import torch
    out = str(tmp_path / "w.bin")
    cmd = [sys.executable, "-m", "paper_2404_02521_gb300.pino_train", "--out", out, "--M", "64",
           "--slices", "8", "--fine-dtau", str(1.0 / 2048), "--problems", "8", "--iters", "30",
           "--batch", "4"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    errs = [float(v) for v in re.findall(r"N=8: ([0-9.eE+-]+|nan|inf)", r.stdout)]
    assert errs and all(np.isfinite(errs)), r.stdout[-2000:]
    net = bs.Pino(out)
    try:
        M, p = 64, PARAMS[0]
        g = bs.Grid(M, 4.0)
        X, Y = fd.mesh(M, 4.0)
        u0 = to_gpu(fd.payoff(p, X, Y))
        u1 = torch.empty_like(u0)
        bs.coarse_propagate(g, bs.COARSE_PINO, net, p, u0, u1, 0.0, 1.0 / 8, 1)
        torch.cuda.synchronize()
        assert torch.isfinite(u1).all()
    finally:
        net.close()


def test_physics_loss_of_a_large_batch(bs):
    # more samples than one launch carries: the library splits the batch
    import torch
    M, B = 24, 40
    rng = np.random.default_rng(9)
    g = bs.Grid(M, 4.0)
    ps = [PARAMS[b % 3] for b in range(B)]
    dts = [0.01 * (1 + b % 5) for b in range(B)]
    prev = [np.asarray(wl.random_field(rng, M), dtype=np.float32) for _ in range(B)]
    pred = [np.asarray(a + 0.01 * wl.random_field(rng, M), dtype=np.float32) for a in prev]
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    bs.pino_physics_loss(g, ps, [to_gpu(a) for a in pred], [to_gpu(a) for a in prev], dts, loss)
    torch.cuda.synchronize()
    got = loss.cpu().numpy()
    for b in range(B):
        p = ps[b]
        w = fd.stencil_weights(M, 4.0, p.sigma1, p.sigma2, p.rho, p.r)
        want = physics.loss(pred[b].astype(np.float64), prev[b].astype(np.float64), dts[b], w)
        assert abs(got[b] - want) <= PHYS_REL_TOL * want, b
