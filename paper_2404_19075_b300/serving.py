"""Replay of a query stream against the library's query server.

Each query is submitted once its (simulated) arrival time has passed and
the server admits it; the loop keeps launching batches and records, for
every query, the wall-clock time from arrival to the moment its completion
is observed. Query kinds follow Sec. V (inference from the trained network):
axial time slices and sub-volumes as grids, and re-projections at any angle
and time.
"""
from __future__ import annotations

import time

import numpy as np
import torch


def request_args(q):
    """(kind, keyword arguments, number of outputs, samples) of a query with
    fields kind, size, t, theta, z, box_lo, box_hi (the seeded stream)."""
    if q.kind == "slice":
        s = q.size
        kw = dict(t=q.t, lo=(-1.0, -1.0, q.z - 1e-3), hi=(1.0, 1.0, q.z + 1e-3), dims=(s, s, 1))
        return "grid", kw, s * s, s * s
    if q.kind == "subvolume":
        s = q.size
        kw = dict(t=q.t, lo=q.box_lo, hi=q.box_hi, dims=(s, s, s))
        return "grid", kw, s ** 3, s ** 3
    S = getattr(q, "S", 256)
    kw = dict(t=q.t, theta=q.theta, rows=q.size, cols=q.size, S=S)
    return "project", kw, q.size * q.size, q.size * q.size * S


def run(model, queries, time_limit=120.0, keep_outputs=False):
    """Replay `queries` (sorted by arrival). Returns a dict with latencies
    (seconds), outputs/s, samples/s, the wall time and, optionally, the
    output tensors by query index."""
    order = sorted(range(len(queries)), key=lambda i: queries[i].arrival)
    pending = list(order)
    inflight = {}
    lat = np.full(len(queries), np.nan)
    outs = {}
    n_out = n_smp = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while pending or inflight:
        now = time.perf_counter() - t0
        if now > time_limit:
            break
        while pending and queries[pending[0]].arrival <= now:
            i = pending[0]
            kind, kw, n, smp = request_args(queries[i])
            out = torch.empty(n, device="cuda")
            rid = model.serve_submit(kind, out, **kw)
            if rid is None:
                break
            inflight[rid] = i
            outs[i] = out
            pending.pop(0)
        model.serve_step()
        done = [rid for rid in list(inflight) if model.serve_poll(rid)]
        tnow = time.perf_counter() - t0
        for rid in done:
            i = inflight.pop(rid)
            lat[i] = tnow - queries[i].arrival
            kind, kw, n, smp = request_args(queries[i])
            n_out += n
            n_smp += smp
            if not keep_outputs:
                outs.pop(i, None)
        if not done and not inflight and pending:
            wait = queries[pending[0]].arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
    wall = time.perf_counter() - t0
    ok = ~np.isnan(lat)
    res = dict(latency=lat, completed=int(ok.sum()), wall=wall,
               outputs_per_s=n_out / wall, samples_per_s=n_smp / wall)
    if ok.any():
        res["p50_ms"] = float(np.percentile(lat[ok], 50) * 1e3)
        res["p99_ms"] = float(np.percentile(lat[ok], 99) * 1e3)
    if keep_outputs:
        res["outputs"] = outs
    return res
