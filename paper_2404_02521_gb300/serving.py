"""Drivers for the serving runtime (bs_server): replay an arrival trace through the server,
and price the same requests one at a time with parareal_solve for comparison.

A request here is any object with .params (workloads.Params-like), .M, .xmax, .N,
.coarse_steps, .tol and an arrival time, and optionally its coarse model: .coarse_kind
(default numerical), .coarse_M (numerical G on that grid; default the request's own) and
.net (a loaded Pino for the PINO G).  Fine steps per slice are chosen by the server's rule
(64, doubled until the Jacobi bound of a fine step is at most 0.7) unless given.
"""
from __future__ import annotations

import time

import numpy as np

from . import _lib


def replay(server: "_lib.Server", reqs, arrivals_s, outputs, fine_steps=None, poll_sleep_s=0.0):
    """Submit reqs[i] at arrivals_s[i] seconds after the start (wall clock) and drive the
    server until every request is done.  Returns (results by request index, makespan in s).
    The latency the server reports runs from submission to completion."""
    order = np.argsort(np.asarray(arrivals_s, dtype=np.float64), kind="stable")
    t0 = time.perf_counter()
    nxt = 0
    by_id = {}
    results = [None] * len(reqs)
    while nxt < len(order) or len(by_id) > 0:
        now = time.perf_counter() - t0
        while nxt < len(order) and arrivals_s[order[nxt]] <= now:
            i = int(order[nxt])
            r = reqs[i]
            fs = 0 if fine_steps is None else int(fine_steps[i])
            rid = server.submit(r.params, r.M, r.xmax, r.N, outputs[i], fine_steps=fs,
                                coarse_steps=r.coarse_steps, tol=r.tol, **coarse_model(r))
            by_id[rid] = i
            nxt += 1
        server.progress()
        for res in server.poll():
            i = by_id.pop(res["id"])
            results[i] = res
        if poll_sleep_s:
            time.sleep(poll_sleep_s)
    return results, time.perf_counter() - t0


def coarse_model(r) -> dict:
    """The request's coarse model as Server.submit keywords."""
    return {"coarse_kind": getattr(r, "coarse_kind", _lib.COARSE_NUM), "coarse_M": getattr(r, "coarse_M", 0),
            "net": getattr(r, "net", None)}


def service_times(reqs, fine_steps, outputs):
    """Each request alone through parareal_solve (with its coarse model), back to back on the
    current stream: device-synchronised wall time per request in ms, iterations and results."""
    import torch
    out = []
    grids = {}
    for i, r in enumerate(reqs):
        cm = coarse_model(r)
        key = (r.M, r.xmax, cm["coarse_M"])
        if key not in grids:
            grids[key] = _lib.Grid(r.M, r.xmax)
            grids[key].set_coarse(cm["coarse_M"])
        g = grids[key]
        U = torch.empty((r.N + 1, r.M, r.M), device="cuda")
        torch.cuda.synchronize()
        t = time.perf_counter()
        pino = cm["coarse_kind"] == _lib.COARSE_PINO
        rc, k, _ = _lib.parareal_solve(g, r.params, r.N, int(fine_steps[i]), cm["coarse_kind"],
                                       1 if pino else r.coarse_steps, cm["net"], r.tol, r.N, U,
                                       allow_maxiter=True)
        outputs[i].copy_(U[r.N])
        torch.cuda.synchronize()
        out.append({"ms": 1e3 * (time.perf_counter() - t), "iterations": k, "status": rc})
        del U
    return out


def fifo_latencies(arrivals_s, service_ms):
    """Latencies (ms) of a single FIFO server that runs one request at a time."""
    order = np.argsort(np.asarray(arrivals_s, dtype=np.float64), kind="stable")
    end = 0.0
    lat = np.zeros(len(order))
    for i in order:
        start = max(end, 1e3 * arrivals_s[i])
        end = start + service_ms[i]
        lat[i] = end - 1e3 * arrivals_s[i]
    return lat, end / 1e3


def shard(n_requests: int, rank: int, world: int):
    """Indices of the requests a replica serves when requests are partitioned across
    world replicas by arrival order (round robin): disjoint, and together all of them."""
    return list(range(rank, n_requests, world))
