"""Continuous-batching request loop over the batching engine.

Requests -- forward modelling, Born modelling or misfit + gradient, each on its own grid --
arrive over time.  Every request that has arrived is submitted to the engine at once; the
engine admits it as soon as its workspace fits into the free part of the device arena
(first-in first-out) and advances it one time step per iteration together with everything
else that runs, so new requests overlap on the GPU with older ones.  Wavefields,
checkpoints and histories stay in the arena for the life of a request; only a request's
inputs go to the device (at submission, on the engine's stream) and its outputs stay there
until the caller reads them.

The loop records, per request, the arrival time, the submission time and the time its
result was complete on the device (observed by the engine's completion event), and reports
throughput and latency percentiles.  A request may carry a deadline: when it has not
finished that long after its arrival, the loop cancels it in the engine (queued or running),
its workspace returns to the arena and its result is dropped; the others are unaffected.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import engine as E
from . import fwi as F


@dataclasses.dataclass
class Request:
    kind: int                    # engine.JOB_MODEL / JOB_BORN / JOB_GRADIENT
    workload: object             # inputs.Workload (grid, model, acquisition, wavelet)
    dxi: tuple | None = None     # Born perturbation (host arrays)
    data: object = None          # gradient: observed traces (host array)
    work_budget: int | None = None   # None: the serving loop's default budget
    deadline_s: float | None = None  # cancel when not done this long after arrival


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def stage(req: Request):
    """Pinned host copies of a request's inputs (what a client would hand over)."""
    w = req.workload
    st = dict(a=_pinned(w.xi_a), b=_pinned(w.xi_b), src=_pinned(w.src_xy), wav=_pinned(w.wavelet),
              rec=_pinned(w.rec_xy))
    if req.dxi is not None:
        st["da"], st["db"] = _pinned(req.dxi[0]), _pinned(req.dxi[1])
    if req.data is not None:
        st["data"] = _pinned(req.data)
    return st


def _submit(eng: E.Engine, req: Request, st, budget):
    w = req.workload
    g = F.make_grid(**w.grid_kwargs())
    dev = lambda t: t.to("cuda", non_blocking=True)
    with torch.cuda.stream(eng.stream):
        a, b, src, wav, rec = dev(st["a"]), dev(st["b"]), dev(st["src"]), dev(st["wav"]), dev(st["rec"])
        if req.kind == E.JOB_MODEL:
            return eng.submit_model(g, w.pz, a, b, src, wav, rec, work_budget=budget)
        if req.kind == E.JOB_BORN:
            return eng.submit_born(g, w.pz, a, b, dev(st["da"]), dev(st["db"]), src, wav, rec, work_budget=budget)
        return eng.submit_gradient(g, w.pz, a, b, src, wav, rec, dev(st["data"]), work_budget=budget)


def default_budget(arena_bytes):
    """Workspace budget of a request: a 16th of the arena, so that all of a request's shots
    run as one group when they fit (fewer, larger steps) while 16 large requests still
    share the arena."""
    return arena_bytes // 16


def serve(requests, arrivals, arena_bytes, iterations_per_call=8, keep_results=False):
    """Runs the request stream: request k arrives at arrivals[k] seconds after the start.
    Returns (stats, results) -- results[k] is the engine Result of request k when
    keep_results, else None."""
    eng = E.Engine(arena_bytes)
    budget = default_budget(arena_bytes)
    staged = [stage(r) for r in requests]
    torch.cuda.synchronize()
    n = len(requests)
    t_sub = np.full(n, np.nan)
    t_done = np.full(n, np.nan)
    ticket_of = {}
    results = [None] * n
    cancelled = np.zeros(n, bool)
    nxt = 0
    t0 = time.perf_counter()
    launches = 0
    max_running = 0
    while nxt < n or ticket_of:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            r = requests[nxt]
            ticket_of[_submit(eng, r, staged[nxt], budget if r.work_budget is None else r.work_budget)] = nxt
            t_sub[nxt] = time.perf_counter() - t0
            nxt += 1
        for t, k in list(ticket_of.items()):    # requests past their deadline
            dl = requests[k].deadline_s
            if dl is not None and now - arrivals[k] > dl:
                eng.cancel(t)
                del ticket_of[t]
                cancelled[k] = True
        if not ticket_of:                       # idle until the next arrival
            if nxt < n:
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            continue
        for res in eng.run(iterations_per_call):
            k = ticket_of.pop(res.ticket)
            t_done[k] = time.perf_counter() - t0
            if keep_results:
                results[k] = res
        launches += F.launch_count()
        max_running = max(max_running, eng.info()["running"])
    wall = time.perf_counter() - t0
    eng.close()
    ok = ~cancelled
    lat = (t_done - arrivals[:n])[ok]
    nok = int(ok.sum())
    stats = dict(requests=n, wall_s=wall, req_per_s=nok / wall,
                 p50_ms=float(np.percentile(lat, 50) * 1e3) if nok else float("nan"),
                 p99_ms=float(np.percentile(lat, 99) * 1e3) if nok else float("nan"),
                 mean_queue_ms=float(np.mean(t_sub - arrivals[:n]) * 1e3), launches=launches,
                 max_running=max_running, cancelled=int(cancelled.sum()))
    return stats, results
