"""Pins for the FP64 FNO / PINO oracle (oracle/fno.py, Sec. 3.4-3.5)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import fd
from oracle import fno


def plane(M, a, b, phase=0.0):
    y, x = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    return np.cos(2 * math.pi * (a * x + b * y) / M + phase)


@pytest.mark.parametrize("a,b", [(1, 0), (3, 2), (11, 5), (4, 11), (2, 28), (7, 21)])
def test_spectral_conv_plane_wave(a, b):
    # For 0 < kx < M/2 a single mode cos(theta) maps to Re(R) cos(theta) - Im(R) sin(theta):
    # pins mode indexing (ky >= M - my stored after ky < my), truncation and the 1/M^2 scale.
    M, mx, my, C = 32, 12, 12, 3
    rng = np.random.default_rng(a * 100 + b)
    R = rng.standard_normal((2 * my, mx, C, 2)) + 1j * rng.standard_normal((2 * my, mx, C, 2))
    v = np.zeros((C, M, M))
    c = 1
    v[c] = plane(M, a, b)
    out = fno.spectral_conv(v, R, mx, my)
    q = b if b < my else b - (M - 2 * my)
    theta = 2 * math.pi * (a * np.arange(M)[None, :] + b * np.arange(M)[:, None]) / M
    for o in range(2):
        want = R[q, a, c, o].real * np.cos(theta) - R[q, a, c, o].imag * np.sin(theta)
        assert np.max(np.abs(out[o] - want)) < 1e-12


@pytest.mark.parametrize("b", [1, 3, 11])
def test_spectral_conv_kx_zero_uses_both_ky(b):
    # cos(2 pi b y / M) has coefficients at ky = b and ky = M - b in the kx = 0 column:
    # out = (Re(R_b + R_-b) cos + (Im(R_-b) - Im(R_b)) sin) / 2
    M, mx, my = 32, 12, 12
    rng = np.random.default_rng(b)
    R = rng.standard_normal((2 * my, mx, 1, 1)) + 1j * rng.standard_normal((2 * my, mx, 1, 1))
    v = plane(M, 0, b)[None]
    out = fno.spectral_conv(v, R, mx, my)[0]
    Rp, Rm = R[b, 0, 0, 0], R[2 * my - b, 0, 0, 0]
    th = 2 * math.pi * b * np.arange(M)[:, None] / M + 0 * np.arange(M)[None, :]
    want = 0.5 * ((Rp.real + Rm.real) * np.cos(th) + (Rm.imag - Rp.imag) * np.sin(th))
    assert np.max(np.abs(out - want)) < 1e-12


@pytest.mark.parametrize("a,b", [(12, 0), (13, 4), (3, 12), (5, 19), (16, 16)])
def test_dropped_modes_vanish(a, b):
    M, mx, my = 32, 12, 12
    R = np.ones((2 * my, mx, 1, 1), dtype=np.complex128)
    out = fno.spectral_conv(plane(M, a, b)[None], R, mx, my)
    assert np.max(np.abs(out)) < 1e-12


def test_spectral_conv_translation_equivariant():
    M, mx, my, C = 32, 6, 5, 4
    rng = np.random.default_rng(7)
    R = rng.standard_normal((2 * my, mx, C, C)) + 1j * rng.standard_normal((2 * my, mx, C, C))
    v = rng.standard_normal((C, M, M))
    a = fno.spectral_conv(np.roll(v, (3, 5), axis=(1, 2)), R, mx, my)
    b = np.roll(fno.spectral_conv(v, R, mx, my), (3, 5), axis=(1, 2))
    assert np.max(np.abs(a - b)) < 1e-10


def test_zero_spectral_weights_is_pointwise_mlp():
    arch = wl.PinoArch(width=8, modes_x=4, modes_y=4, layers=2, proj_hidden=16)
    w = wl.pino_random_weights(arch, seed=3)
    w["spec_w"][:] = 0
    M = 24
    rng = np.random.default_rng(0)
    a = rng.standard_normal((arch.in_channels, M, M))
    out = fno.fno_forward(a, w, arch.modes_x, arch.modes_y)
    j, i = 5, 17
    h = a[:, j, i] @ w["lift_w"] + w["lift_b"]
    for l in range(arch.layers):
        h = np.maximum(h @ w["pw_w"][l] + w["pw_b"][l], 0)
    z = np.maximum(h @ w["proj1_w"] + w["proj1_b"], 0)
    assert abs(out[j, i] - (z @ w["proj2_w"] + w["proj2_b"])) < 1e-12


def test_bilinear_resample_exact_on_bilinear_functions():
    for Mi, Mo in [(33, 9), (9, 33), (1024, 256), (256, 1024), (17, 17)]:
        X, Y = fd.mesh(Mi, 4.0)
        f = lambda X, Y: 0.3 + 1.7 * X - 0.4 * Y + 0.25 * X * Y
        Xo, Yo = fd.mesh(Mo, 4.0)
        got = fno.bilinear_resample(f(X, Y), Mo)
        assert np.max(np.abs(got - f(Xo, Yo))) < 1e-11


def test_pino_coarse_sets_far_field():
    arch = wl.PinoArch(width=8, modes_x=4, modes_y=4, layers=1, proj_hidden=8)
    w = wl.pino_random_weights(arch, seed=1)
    p = wl.exchange_cfg2(0.7).params
    M = 24
    X, Y = fd.mesh(M, 4.0)
    u = fd.payoff(p, X, Y)
    out = fno.pino_coarse(u, 4.0, 0.25, 0.125, p, w, arch.modes_x, arch.modes_y)
    g = fd.dirichlet(p)(X, Y, 0.375)
    assert np.array_equal(out[M - 1], g[M - 1]) and np.array_equal(out[:, M - 1], g[:, M - 1])
