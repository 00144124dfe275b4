"""ctypes binding of libbsparareal.so: argument marshalling only.

Every function mirrors an entry point of include/bsparareal.h and takes torch tensors (or
raw device pointers) for device arrays.  All arithmetic happens in the CUDA library; if the
library cannot be loaded this module raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbsparareal.so")

BS_OK, BS_ERR_ARG, BS_ERR_CUDA, BS_ERR_NOCONV, BS_ERR_MAXITER, BS_ERR_OOM, BS_ERR_FILE = 0, -1, -2, -3, -4, -5, -6
ERR_NAMES = {0: "BS_OK", -1: "BS_ERR_ARG", -2: "BS_ERR_CUDA", -3: "BS_ERR_NOCONV",
             -4: "BS_ERR_MAXITER", -5: "BS_ERR_OOM", -6: "BS_ERR_FILE"}
BASKET, EXCHANGE, CALL1, CASH_OR_NOTHING = 0, 1, 2, 3
COARSE_NUM, COARSE_PINO = 0, 1

# exported entry points declared in include/bsparareal.h
EXPORTS = ["bs_last_error", "bs_grid_create", "bs_grid_destroy", "bs_payoff",
           "fine_propagate_batched", "coarse_propagate", "pino_load", "pino_destroy",
           "parareal_solve", "bs_fine_sweeps", "bs_set_option", "bs_grid_stats", "bs_phase_stats", "parareal_solve_noalloc",
           "bs_coarse_variant", "bs_coarse_variant_info", "bs_payoff3", "fine_propagate3", "coarse_propagate3", "parareal_solve3", "bs_server_create", "bs_server_submit", "bs_server_progress",
           "bs_server_poll", "bs_server_stats", "bs_server_destroy", "bs_fine_steps_for",
           "bs_grid_set_coarse", "bs_device_allocations", "parareal_sweep_range", "coarse_propagate_batched",
           "pino_physics_loss"]
OPT_FINE_SWEEPS, OPT_JACOBI_TARGET, OPT_KRYLOV_TOL, OPT_KRYLOV_MAXIT, OPT_PHASE_TIMING = 0, 1, 2, 3, 4
OPT_JACOBI_TARGET_COLD = 5
OPT_COARSE_VARIANT = 6
OPT_JACOBI_TARGET_EXTRAP = 7
OPT_EXTRAP_START = 8
OPT_EXTRAP_LATE = 9
OPT_JACOBI_TARGET_EXTRAP_LATE = 10
OPT_PIPELINE = 11
OPT_FINE_KRYLOV_TOL = 12
OPT_FINE_TILE = 13
PARAREAL_USER_U0 = 0x100


class bs_params(C.Structure):
    _fields_ = [("sigma1", C.c_double), ("sigma2", C.c_double), ("rho", C.c_double),
                ("r", C.c_double), ("T", C.c_double), ("strike", C.c_double),
                ("w1", C.c_double), ("w2", C.c_double), ("payoff", C.c_int),
                ("reserved", C.c_int), ("strike2", C.c_double), ("cash", C.c_double)]


class bs_params3(C.Structure):
    _fields_ = [("sigma", C.c_double * 3), ("rho", C.c_double * 3), ("r", C.c_double),
                ("strike", C.c_double), ("w", C.c_double * 3), ("payoff", C.c_int),
                ("reserved", C.c_int)]


class bs_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int)]


class bs_request(C.Structure):
    _fields_ = [("p", bs_params), ("M", C.c_int), ("xmax", C.c_double), ("N", C.c_int),
                ("fine_steps", C.c_int), ("coarse_steps", C.c_int), ("tol", C.c_double),
                ("Kmax", C.c_int), ("u_out", C.c_void_p), ("coarse_kind", C.c_int), ("coarse_M", C.c_int),
                ("net", C.c_void_p)]


class bs_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("iterations", C.c_int),
                ("defect", C.c_double), ("latency_ms", C.c_double), ("fine_steps", C.c_int)]


class bs_server_stats_t(C.Structure):
    _fields_ = [("arena_bytes", C.c_size_t), ("arena_used", C.c_size_t),
                ("fine_batches", C.c_longlong), ("fine_items", C.c_longlong),
                ("coarse_sweeps", C.c_longlong), ("launches", C.c_longlong)]


class BSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: Optional[str] = None):
    """Load the shared library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if path is None:
        if not _build.up_to_date():
            _build.build()
        path = LIB_PATH
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    lib.bs_last_error.restype = C.c_char_p
    lib.bs_last_error.argtypes = []
    lib.bs_grid_create.argtypes = [i, d, P(vp)]
    lib.bs_grid_destroy.argtypes = [vp]
    lib.bs_payoff.argtypes = [vp, P(bs_params), vp, vp]
    lib.fine_propagate_batched.argtypes = [vp, P(bs_params), P(vp), P(vp), P(d), P(d), i, i, vp]
    lib.coarse_propagate.argtypes = [vp, i, vp, P(bs_params), vp, vp, d, d, i, vp]
    lib.pino_load.argtypes = [C.c_char_p, P(vp)]
    lib.pino_physics_loss.argtypes = [vp, P(bs_params), P(vp), P(vp), P(d), i, vp, P(vp), vp]
    lib.pino_destroy.argtypes = [vp]
    lib.parareal_solve.argtypes = [vp, P(bs_params), i, i, i, i, vp, d, i, vp, P(i), P(d), vp]
    lib.bs_fine_sweeps.argtypes = [vp, P(bs_params), d, i]
    lib.bs_set_option.argtypes = [i, d]
    lib.bs_grid_stats.argtypes = [vp, P(i), P(i), P(i), P(i)]
    lib.bs_coarse_variant.argtypes = [vp, P(bs_params), d, P(i), vp]
    lib.bs_coarse_variant_info.argtypes = [i, i, P(i), P(i), P(i), P(i), P(i)]
    lib.bs_payoff3.argtypes = [i, d, P(bs_params3), vp, vp]
    lib.fine_propagate3.argtypes = [i, d, P(bs_params3), P(vp), P(vp), P(d), i, d, i, vp]
    lib.coarse_propagate3.argtypes = [i, d, P(bs_params3), vp, vp, d, d, i, vp]
    lib.parareal_solve3.argtypes = [i, d, P(bs_params3), d, i, i, i, d, i, vp, P(i), P(d), vp]
    lib.bs_server_create.argtypes = [P(bs_server_config), P(vp)]
    lib.bs_server_submit.argtypes = [vp, P(bs_request), P(C.c_longlong)]
    lib.bs_server_progress.argtypes = [vp, P(i), P(i)]
    lib.bs_server_poll.argtypes = [vp, P(bs_result), i, P(i)]
    lib.bs_server_stats.argtypes = [vp, P(bs_server_stats_t)]
    lib.bs_server_destroy.argtypes = [vp]
    lib.bs_fine_steps_for.argtypes = [i, P(bs_params), i, i, d, P(i)]
    lib.bs_grid_set_coarse.argtypes = [vp, i]
    lib.bs_phase_stats.argtypes = [vp, P(d), P(i), P(d), P(i), P(i)]
    lib.parareal_solve_noalloc.argtypes = [i, d, P(bs_params), i, i, i, d, i, vp, P(i), P(d), vp]
    lib.bs_device_allocations.argtypes = [P(C.c_longlong)]
    lib.parareal_sweep_range.argtypes = [vp, P(bs_params), i, i, i, i, i, vp, vp, vp, vp, vp]
    lib.coarse_propagate_batched.argtypes = [vp, i, vp, P(bs_params), P(vp), P(vp), P(d), d, i, i, vp]
    for name in EXPORTS:
        if name != "bs_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().bs_last_error().decode()


def check(rc: int, allow=()) -> int:
    if rc != BS_OK and rc not in allow:
        raise BSError(rc, last_error())
    return rc


def to_params(p) -> bs_params:
    """From a workloads.Params-like object (attributes sigma1 ... cash)."""
    return bs_params(float(p.sigma1), float(p.sigma2), float(p.rho), float(p.r), float(p.T),
                     float(p.strike), float(p.w1), float(p.w2), int(p.payoff), 0,
                     float(getattr(p, "strike2", 0.0)), float(getattr(p, "cash", 1.0)))


def to_params3(p) -> bs_params3:
    """From an object with sigma (3), rho (rho_12, rho_13, rho_23), r, strike, w (3), payoff."""
    return bs_params3((C.c_double * 3)(*[float(v) for v in p.sigma]),
                      (C.c_double * 3)(*[float(v) for v in p.rho]), float(p.r),
                      float(getattr(p, "strike", 1.0)),
                      (C.c_double * 3)(*[float(v) for v in getattr(p, "w", (1 / 3, 1 / 3, 1 / 3))]),
                      int(p.payoff), 0)


def _ptr(x) -> int:
    return x if isinstance(x, int) else x.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Grid:
    """bs_grid handle: M x M nodes on [0, xmax]^2."""

    def __init__(self, M: int, xmax: float):
        lib = load()
        h = C.c_void_p()
        check(lib.bs_grid_create(int(M), float(xmax), C.byref(h)))
        self.h, self.M, self.xmax = h, int(M), float(xmax)

    def set_coarse(self, Mc: int):
        """Run the numerical coarse propagator on an Mc x Mc grid with bilinear resampling
        (0: on this grid)."""
        check(load().bs_grid_set_coarse(self.h, int(Mc)))

    def close(self):
        if self.h:
            load().bs_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bs_payoff(g: Grid, p, u, stream=None):
    bp = to_params(p)
    return check(load().bs_payoff(g.h, C.byref(bp), _ptr(u), _stream(stream)))


def fine_propagate_batched(g: Grid, params: Sequence, u_in: Sequence, u_out: Sequence,
                           tau0: Sequence[float], dtau: Sequence[float], nsteps: int,
                           stream=None):
    B = len(u_in)
    P = (bs_params * B)(*[to_params(p) for p in params])
    pin = (C.c_void_p * B)(*[_ptr(x) for x in u_in])
    pout = (C.c_void_p * B)(*[_ptr(x) for x in u_out])
    t0 = (C.c_double * B)(*[float(t) for t in tau0])
    dt = (C.c_double * B)(*[float(t) for t in dtau])
    return check(load().fine_propagate_batched(g.h, P, pin, pout, t0, dt, int(nsteps), B,
                                               _stream(stream)))


def pino_physics_loss(g: Grid, params: Sequence, u_pred: Sequence, u_prev: Sequence,
                      dtau: Sequence[float], loss, grad: Optional[Sequence] = None, stream=None):
    """PDE term of the PINO training loss (Sec. 3.5): loss[b] (a device float64 tensor of
    len(u_pred)) and, with grad, d loss[b] / d u_pred[b] into grad[b]."""
    B = len(u_pred)
    P = (bs_params * B)(*[to_params(p) for p in params])
    pp = (C.c_void_p * B)(*[_ptr(x) for x in u_pred])
    pv = (C.c_void_p * B)(*[_ptr(x) for x in u_prev])
    dt = (C.c_double * B)(*[float(t) for t in dtau])
    pg = (C.c_void_p * B)(*[_ptr(x) for x in grad]) if grad is not None else None
    return check(load().pino_physics_loss(g.h, P, pp, pv, dt, B, _ptr(loss), pg, _stream(stream)))


def bs_payoff3(M: int, xmax: float, p, u, stream=None):
    """Three-asset payoff into a device float[M^3] tensor."""
    bp = to_params3(p)
    return check(load().bs_payoff3(int(M), float(xmax), C.byref(bp), _ptr(u), _stream(stream)))


def fine_propagate3(M: int, xmax: float, p, u_in: Sequence, u_out: Sequence, tau0: Sequence[float],
                    dtau: float, nsteps: int, stream=None):
    """F for three assets (19-point stencil) on len(u_in) states of M^3 nodes."""
    bp = to_params3(p)
    B = len(u_in)
    pin = (C.c_void_p * B)(*[_ptr(x) for x in u_in])
    pout = (C.c_void_p * B)(*[_ptr(x) for x in u_out])
    t0 = (C.c_double * B)(*[float(t) for t in tau0])
    return check(load().fine_propagate3(int(M), float(xmax), C.byref(bp), pin, pout, t0, B, float(dtau),
                                        int(nsteps), _stream(stream)))


def coarse_propagate3(M: int, xmax: float, p, u_in, u_out, tau0: float, dtau_slice: float, nsteps: int,
                      stream=None):
    """Three-asset G: nsteps BiCGSTAB-solved implicit steps over dtau_slice (synchronous)."""
    bp = to_params3(p)
    return check(load().coarse_propagate3(int(M), float(xmax), C.byref(bp), _ptr(u_in), _ptr(u_out),
                                          float(tau0), float(dtau_slice), int(nsteps), _stream(stream)))


def parareal_solve3(M: int, xmax: float, p, T: float, N: int, fine_steps: int, coarse_steps: int,
                    tol: float, Kmax: int, u_out, stream=None, allow_maxiter=True):
    """Three-asset Parareal.  Returns (status, k_done, defects)."""
    bp = to_params3(p)
    k = C.c_int(0)
    hist = (C.c_double * max(1, Kmax))()
    rc = load().parareal_solve3(int(M), float(xmax), C.byref(bp), float(T), int(N), int(fine_steps),
                                int(coarse_steps), float(tol), int(Kmax), _ptr(u_out), C.byref(k), hist,
                                _stream(stream))
    check(rc, allow=(BS_ERR_MAXITER,) if allow_maxiter else ())
    return rc, k.value, [hist[i] for i in range(k.value)]


def coarse_propagate(g: Grid, kind: int, net, p, u_in, u_out, tau0: float, dtau_slice: float,
                     nsteps: int, stream=None):
    bp = to_params(p)
    return check(load().coarse_propagate(g.h, int(kind), net.h if net is not None else None,
                                         C.byref(bp), _ptr(u_in), _ptr(u_out), float(tau0),
                                         float(dtau_slice), int(nsteps), _stream(stream)))


def parareal_solve(g: Grid, p, N: int, fine_steps: int, coarse_kind: int, coarse_steps: int,
                   net, tol: float, Kmax: int, u_out, stream=None, allow_maxiter=True):
    """Returns (status, k_done, defects)."""
    bp = to_params(p)
    k = C.c_int(0)
    hist = (C.c_double * max(1, Kmax))()
    rc = load().parareal_solve(g.h, C.byref(bp), int(N), int(fine_steps), int(coarse_kind),
                               int(coarse_steps), net.h if net is not None else None,
                               float(tol), int(Kmax), _ptr(u_out), C.byref(k), hist,
                               _stream(stream))
    check(rc, allow=(BS_ERR_MAXITER,) if allow_maxiter else ())
    return rc, k.value, [hist[i] for i in range(k.value)]


def parareal_solve_noalloc(M: int, xmax: float, p, N: int, fine_steps: int, coarse_steps: int,
                           tol: float, Kmax: int, u_out, stream=None, allow_maxiter=True):
    """parareal_solve without device allocation (scratch in a fixed device array).
    Returns (status, k_done, defects)."""
    bp = to_params(p)
    k = C.c_int(0)
    hist = (C.c_double * max(1, Kmax))()
    rc = load().parareal_solve_noalloc(int(M), float(xmax), C.byref(bp), int(N), int(fine_steps),
                                       int(coarse_steps), float(tol), int(Kmax), _ptr(u_out),
                                       C.byref(k), hist, _stream(stream))
    check(rc, allow=(BS_ERR_MAXITER,) if allow_maxiter else ())
    return rc, k.value, [hist[i] for i in range(k.value)]


def coarse_propagate_batched(g: Grid, kind: int, net, params: Sequence, u_in: Sequence, u_out: Sequence,
                             tau0: Sequence[float], dtau_slice: float, nsteps: int = 1, stream=None):
    """G on len(u_in) independent states at once (numerical: nsteps steps; PINO: the network)."""
    B = len(u_in)
    bp = (bs_params * B)(*[to_params(p) for p in params])
    ins = (C.c_void_p * B)(*[_ptr(u) for u in u_in])
    outs = (C.c_void_p * B)(*[_ptr(u) for u in u_out])
    t0 = (C.c_double * B)(*[float(t) for t in tau0])
    return check(load().coarse_propagate_batched(g.h, int(kind), net.h if net is not None else None, bp, ins, outs,
                                                 t0, float(dtau_slice), int(nsteps), B, _stream(stream)))


def parareal_sweep_range(g: Grid, p, N: int, coarse_steps: int, k: int, n_begin: int, n_end: int,
                         U, Fb, Gold, norms, stream=None):
    """The serial coarse sweep over slices [n_begin, n_end) (k = -1: the initial sweep)."""
    bp = to_params(p)
    return check(load().parareal_sweep_range(g.h, C.byref(bp), int(N), int(coarse_steps), int(k),
                                             int(n_begin), int(n_end), _ptr(U),
                                             _ptr(Fb) if Fb is not None else None, _ptr(Gold),
                                             _ptr(norms), _stream(stream)))


def bs_device_allocations() -> int:
    """Device (and pinned host) allocations the library has made in this process."""
    n = C.c_longlong(0)
    check(load().bs_device_allocations(C.byref(n)))
    return n.value


def bs_fine_steps_for(M: int, p, N: int, min_steps: int = 64, qmax: float = 0.7) -> int:
    """Smallest min_steps * 2^k fine steps per slice whose Jacobi bound is <= qmax."""
    bp = to_params(p)
    s = C.c_int(0)
    check(load().bs_fine_steps_for(int(M), C.byref(bp), int(N), int(min_steps), float(qmax), C.byref(s)))
    return s.value


START_WARM, START_COLD, START_EXTRAP, START_EXTRAP_LATE = 0, 1, 2, 3


def bs_fine_sweeps(g: Grid, p, dtau: float, first_step=False) -> int:
    """Jacobi sweeps per fine step; first_step: True/1 = cold first step, False/0 = warm
    start, 2 = extrapolated start, 3 = extrapolated start after the transient."""
    bp = to_params(p)
    return int(load().bs_fine_sweeps(g.h, C.byref(bp), float(dtau), int(first_step)))


def bs_set_option(option: int, value: float):
    return check(load().bs_set_option(int(option), float(value)))


def bs_coarse_variant(g: Grid, p, dtau_coarse: float, stream=None) -> int:
    """Coarse band variant used on this grid (measured on first use; -1 for M > 256)."""
    bp = to_params(p)
    v = C.c_int(-1)
    check(load().bs_coarse_variant(g.h, C.byref(bp), float(dtau_coarse), C.byref(v), _stream(stream)))
    return v.value


def bs_coarse_variant_info(variant: int, M: int) -> dict:
    """Cluster CTAs, threads per CTA, rows per thread and solver features (degree of the
    polynomial preconditioner, 0 for none; quadratic extrapolation) of a band variant on an
    M x M grid (host-only)."""
    v = [C.c_int(0) for _ in range(5)]
    check(load().bs_coarse_variant_info(int(variant), int(M), *[C.byref(x) for x in v]))
    return {"ctas": v[0].value, "threads": v[1].value, "rows": v[2].value, "poly": v[3].value,
            "quad": bool(v[4].value)}


def bs_grid_stats(g: Grid, detail: bool = False):
    """(max BiCGSTAB iterations, any solve hit its cap) since the last reset; with detail,
    also (summed iterations, number of implicit solves)."""
    it, fail, tot, ns = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
    check(load().bs_grid_stats(g.h, C.byref(it), C.byref(fail), C.byref(tot), C.byref(ns)))
    if detail:
        return it.value, bool(fail.value), tot.value, ns.value
    return it.value, bool(fail.value)


def bs_phase_stats(g: Grid) -> dict:
    """Launch counts and (with OPT_PHASE_TIMING) event-timed ms per phase; resets them."""
    fm, cm = C.c_double(0), C.c_double(0)
    fl, cl, ol = C.c_int(0), C.c_int(0), C.c_int(0)
    check(load().bs_phase_stats(g.h, C.byref(fm), C.byref(fl), C.byref(cm), C.byref(cl), C.byref(ol)))
    return {"fine_ms": fm.value, "fine_launches": fl.value, "coarse_ms": cm.value,
            "coarse_launches": cl.value, "other_launches": ol.value}


class Pino:
    """bs_pino handle loaded from a weight file."""

    def __init__(self, path: str):
        h = C.c_void_p()
        check(load().pino_load(path.encode(), C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            load().pino_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """bs_server handle: continuous batching of Parareal requests (each with its coarse model)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 32):
        cfg = bs_server_config(int(hbm_budget_bytes), int(max_active))
        h = C.c_void_p()
        check(load().bs_server_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self._keep = {}   # id -> output buffer kept alive until the request is done

    def submit(self, p, M, xmax, N, u_out, fine_steps=0, coarse_steps=1, tol=1e-4, Kmax=None,
               coarse_kind=COARSE_NUM, coarse_M=0, net=None) -> int:
        r = bs_request(to_params(p), int(M), float(xmax), int(N), int(fine_steps), int(coarse_steps),
                       float(tol), int(N if Kmax is None else Kmax), _ptr(u_out), int(coarse_kind),
                       int(coarse_M), net.h if net is not None else None)
        rid = C.c_longlong(0)
        check(load().bs_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (u_out, net)
        return rid.value

    def progress(self):
        a, q = C.c_int(0), C.c_int(0)
        check(load().bs_server_progress(self.h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, max_results: int = 256):
        buf = (bs_result * max_results)()
        n = C.c_int(0)
        check(load().bs_server_poll(self.h, buf, int(max_results), C.byref(n)))
        out = []
        for k in range(n.value):
            r = buf[k]
            self._keep.pop(r.id, None)
            out.append({"id": r.id, "status": r.status, "iterations": r.iterations, "defect": r.defect,
                        "latency_ms": r.latency_ms, "fine_steps": r.fine_steps})
        return out

    def stats(self) -> dict:
        st = bs_server_stats_t()
        check(load().bs_server_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in bs_server_stats_t._fields_}

    def close(self):
        if self.h:
            load().bs_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
