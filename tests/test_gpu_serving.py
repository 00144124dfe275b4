"""Serving runtime (bs_server): continuous batching of Parareal requests of different grid
sizes and slice counts.  Each result must be the same alone and in the mix (bitwise: every
slice of a batched fine launch and every coarse sweep is computed independently of the other
requests), admission must respect the HBM budget, and the results must be the Parareal
solutions the oracle defines."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_util import rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    import paper_2404_02521_gb300 as bs
    bs.load()
    return bs


def mix():
    rng = np.random.default_rng(7)
    out = []
    for k, (M, N) in enumerate([(40, 4), (64, 8), (100, 4), (64, 6), (300, 4), (33, 8), (128, 4)]):
        payoff = wl.BASKET if k % 2 == 0 else wl.EXCHANGE
        p = wl.random_params(rng, payoff, float(rng.uniform(0.25, 1.0)))
        out.append(wl.Problem(f"mix{k}", M, 4.0, N, 0, 1, p))
    return out


def alone(bs, reqs):
    """Each request through a server on its own (nothing else on the device)."""
    import torch
    from paper_2404_02521_gb300 import serving
    outs = [torch.empty((r.M, r.M), device="cuda") for r in reqs]
    sv = bs.Server(1 << 30, 8)
    for i, r in enumerate(reqs):
        serving.replay(sv, [r], [0.0], [outs[i]])
    sv.close()
    return outs


def plain(bs, reqs, fine_steps):
    """Each request through parareal_solve, F and the sweep alternating (the algorithm the
    server runs per request)."""
    import torch
    from paper_2404_02521_gb300 import serving
    outs = [torch.empty((r.M, r.M), device="cuda") for r in reqs]
    try:
        bs.bs_set_option(bs.OPT_PIPELINE, 0)
        serving.service_times(reqs, fine_steps, outs)
    finally:
        bs.bs_set_option(bs.OPT_PIPELINE, 1)
    return outs


def test_mix_switches_fine_layouts_bitwise(bs):
    # two 256^2 requests with the same parameters share their F launches in the mix (16
    # states: the 8-CTA band layout) but not alone (8 states: the 16-CTA layout), and a 512^2
    # request's F runs as cluster tiles; every result is the same bit for bit either way
    import torch
    from paper_2404_02521_gb300 import serving
    p = wl.exchange_cfg2(0.7).params
    reqs = [wl.Problem("s256a", 256, 4.0, 8, 0, 1, p), wl.Problem("s256b", 256, 4.0, 8, 0, 1, p),
            wl.Problem("s512", 512, 4.0, 4, 0, 1, wl.basket_cfg1().params)]
    outs = [torch.zeros((r.M, r.M), device="cuda") for r in reqs]
    sv = bs.Server(1 << 31, 4)
    res, _ = serving.replay(sv, reqs, [0.0, 0.0, 0.0], outs)
    sv.close()
    assert all(r["status"] == 0 for r in res), res
    assert torch.equal(outs[0], outs[1])
    for r, a, b in zip(reqs, outs, alone(bs, reqs)):
        assert torch.equal(a, b), r.name


def test_mix_equals_alone_bitwise(bs):
    import torch
    from paper_2404_02521_gb300 import serving
    reqs = mix()
    outs = [torch.zeros((r.M, r.M), device="cuda") for r in reqs]
    sv = bs.Server(1 << 30, 8)
    # two waves: the second arrives while the first is on the GPU
    arrivals = [0.0, 0.0, 0.0, 0.0, 0.01, 0.01, 0.02]
    res, _ = serving.replay(sv, reqs, arrivals, outs)
    st = sv.stats()
    sv.close()
    assert all(r["status"] == 0 for r in res), res
    assert st["arena_used"] == 0 and st["fine_batches"] >= 1
    fs = [r["fine_steps"] for r in res]
    for r, a, b, c in zip(reqs, outs, alone(bs, reqs), plain(bs, reqs, fs)):
        assert torch.equal(a, b), r.name
        assert torch.equal(a, c), r.name


def test_admission_waits_for_memory(bs):
    # a budget that holds about two of the requests: the others wait and still finish
    import torch
    from paper_2404_02521_gb300 import serving
    reqs = [wl.Problem(f"b{k}", 128, 4.0, 8, 0, 1, wl.basket_cfg1().params) for k in range(6)]
    need = (3 * 8 + 1) * 128 * 128 * 4 + 16 * 9
    sv = bs.Server(2 * need + 4096, 8)
    outs = [torch.zeros((128, 128), device="cuda") for _ in reqs]
    res, _ = serving.replay(sv, reqs, [0.0] * len(reqs), outs)
    sv.close()
    assert all(r["status"] == 0 for r in res)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_serving_result_is_parareal_solution(bs):
    # the served price surface equals the oracle's Parareal solution within the coarse
    # tolerance and the serial fine solution within the Parareal tolerance
    import torch
    from oracle import fd
    from oracle import parareal as opr
    from paper_2404_02521_gb300 import serving
    pb = wl.Problem("srv", 40, 4.0, 6, 0, 1, wl.basket_cfg1().params)
    out = torch.zeros((40, 40), device="cuda")
    sv = bs.Server(1 << 28, 2)
    res, _ = serving.replay(sv, [pb], [0.0], [out])
    sv.close()
    fs = res[0]["fine_steps"]
    pbf = wl.Problem("srv", 40, 4.0, 6, fs, 1, pb.params)
    F = fd.SlicePropagator(40, 4.0, pb.params, 6, fs)
    G = fd.SlicePropagator(40, 4.0, pb.params, 6, 1)
    serial = fd.serial_fine(pbf)
    Uo, ko, _, _ = opr.parareal(serial[0], F, G, 6, 1e-4, 6)
    assert res[0]["iterations"] == ko
    assert rel_err(to_np(out), Uo[6]) <= 6e-5
    assert rel_err(to_np(out), serial[6]) <= 1e-3


def test_long_queue_admits_every_request_intact(bs):
    # many more requests than slots, all queued at once: the pending queue is drained across
    # many of its storage blocks, and every request must be admitted with its own parameters
    # (its result equals the same request solved alone)
    import torch
    from paper_2404_02521_gb300 import serving
    rng = np.random.default_rng(11)
    reqs = []
    for k in range(96):
        p = wl.random_params(rng, wl.BASKET if k % 2 else wl.EXCHANGE, float(rng.uniform(0.25, 1.0)))
        reqs.append(wl.Problem(f"q{k}", int(rng.choice([16, 24, 32])), 4.0, int(rng.choice([4, 6])), 0, 1, p))
    outs = [torch.zeros((r.M, r.M), device="cuda") for r in reqs]
    sv = bs.Server(1 << 28, 3)
    res, _ = serving.replay(sv, reqs, [0.0] * len(reqs), outs)
    st = sv.stats()
    sv.close()
    assert all(r is not None and r["status"] == 0 for r in res)
    assert st["arena_used"] == 0
    ref = alone(bs, reqs[::8])
    for a, b in zip(outs[::8], ref):
        assert torch.equal(a, b)


def test_coarse_models_mix_equals_alone(bs, tmp_path):
    # requests with the numerical G on their own grid, the numerical G on a coarse grid and
    # the PINO, all in one mix (the PINO sweeps of two requests share the network): each
    # result equals the same request alone through the server and through parareal_solve's
    # phase-by-phase driver with the same coarse model, bit for bit
    import types

    import torch
    from paper_2404_02521_gb300 import pino_io, serving
    arch = wl.PinoArch()
    w = wl.pino_random_weights(arch, seed=23, spectral_scale=8.0)
    w["proj2_w"] = 0.05 * w["proj2_w"]
    w["proj2_b"] = np.float64(0.0)
    path = str(tmp_path / "w.bin")
    pino_io.write_weights(path, w, arch.in_channels, arch.width, arch.modes_x, arch.modes_y, arch.layers,
                          arch.proj_hidden)
    net = bs.Pino(path)
    rng = np.random.default_rng(5)
    specs = [(128, 8, bs.COARSE_NUM, 64), (64, 8, bs.COARSE_PINO, 0), (300, 4, bs.COARSE_NUM, 100),
             (96, 6, bs.COARSE_NUM, 0), (128, 4, bs.COARSE_PINO, 0), (200, 8, bs.COARSE_NUM, 72)]
    reqs = []
    for k, (M, N, kind, Mc) in enumerate(specs):
        p = wl.random_params(rng, wl.BASKET if k % 2 == 0 else wl.EXCHANGE, float(rng.uniform(0.25, 1.0)))
        reqs.append(types.SimpleNamespace(name=f"cm{k}", params=p, M=M, xmax=4.0, N=N, coarse_steps=2, tol=1e-4,
                                          coarse_kind=kind, coarse_M=Mc,
                                          net=net if kind == bs.COARSE_PINO else None))
    outs = [torch.zeros((r.M, r.M), device="cuda") for r in reqs]
    sv = bs.Server(1 << 30, 8)
    res, _ = serving.replay(sv, reqs, [0.0, 0.0, 0.0, 0.005, 0.005, 0.01], outs)
    st = sv.stats()
    sv.close()
    assert all(r["status"] == 0 for r in res), res
    assert st["arena_used"] == 0
    fs = [r["fine_steps"] for r in res]
    for r, a, b, c in zip(reqs, outs, alone(bs, reqs), plain(bs, reqs, fs)):
        assert torch.equal(a, b), r.name
        assert torch.equal(a, c), r.name


def test_submit_rejects_bad_coarse_models(bs):
    import torch
    out = torch.zeros((64, 64), device="cuda")
    p = wl.basket_cfg1().params
    sv = bs.Server(1 << 26, 2)
    try:
        for kw in ({"coarse_kind": 7}, {"coarse_M": 4}, {"coarse_M": 65},
                   {"coarse_kind": bs.COARSE_PINO}):   # the PINO without a network
            with pytest.raises(bs.BSError):
                sv.submit(p, 64, 4.0, 8, out, **kw)
    finally:
        sv.close()
