"""Batching, serving, differentiation, error-bowl and inversion workloads
(bench.py --workload batch|serve|differentiation|bowls|invert).

Each prints one JSON line.  Cell-updates count computational cells (sponge included) x steps
x shots x propagation passes, as bench.py's default line does: forward modelling 1, Born 1
(its background and scattered fields count as one pass), gradient 2 (forward and adjoint;
recomputed forward steps are not counted).
"""
from __future__ import annotations

import json
import time

import numpy as np
import torch

from . import engine as E
from . import fwi as F
from . import inputs as I
from . import serve as S

METRIC = "Gcell-updates/s & FWI gradients/s vs plain per-shot GPU; p50/p99 solve latency"
PASSES = {E.JOB_MODEL: 1, E.JOB_BORN: 1, E.JOB_GRADIENT: 2}
OPS = {E.JOB_MODEL: F.OP_MODEL, E.JOB_BORN: F.OP_BORN, E.JOB_GRADIENT: F.OP_GRADIENT}


def kernel_profile(enable, every=1):
    """Per-kernel device time recorded by the library's launch events (fwi_profile), one launch
    in `every` of each kernel timed; a kernel's time is its timed mean times its launches."""
    import ctypes
    L = F.lib()
    if enable:
        L.fwi_profile(int(every))
        return None
    buf = ctypes.create_string_buffer(1 << 16)
    L.fwi_profile_report(buf, len(buf))
    L.fwi_profile(0)
    prof = {}
    for line in buf.value.decode().splitlines():
        name, seen, cnt, tot = line.rsplit(" ", 3)
        prof[name.replace("fwi::", "").replace("(", "").replace(")", "").replace(", ", ",")] = (
            int(seen), float(tot) / int(cnt) * int(seen))
    total = sum(v[1] for v in prof.values()) or 1.0
    return {"device_ms": round(total, 1),
            "kernels": {k: {"launches": c, "ms": round(t, 1), "share": round(t / total, 4)}
                        for k, (c, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}}


def cells(w):
    return (w.nx + 2 * w.sponge) * (w.nz + 2 * w.sponge) * w.nt * w.ns


def grid_of(w):
    return F.make_grid(**w.grid_kwargs())


def _drain(eng, ticket_jobs):
    """Runs the engine until every ticket is done; returns (wall s, launches, results)."""
    out, launches = {}, 0
    t0 = time.perf_counter()
    while len(out) < len(ticket_jobs):
        for r in eng.run(32):
            out[r.ticket] = r
        launches += F.launch_count()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, launches, out


def run_batch(njobs, Clocks, profile=False, total=256):
    """The first `njobs` of inputs.batch_jobs(total, seed=0) through the engine: their forward
    models (observed data), then their misfit gradients at the background, each phase one engine
    run; against the plain per-shot GPU path on a sample of the same jobs.  Returns a dict."""
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    jobs = I.batch_jobs(total, seed=0)[:njobs]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    staged = [dict(a=d(w.xi_a), b=d(w.xi_b), src=d(w.src_xy), rec=d(w.rec_xy), wav=d(w.wavelet),
                   zero=torch.zeros((w.nz, w.nx), dtype=torch.float32, device=dev)) for w in jobs]
    free, _ = torch.cuda.mem_get_info(dev)
    # leave room for every job's traces and float64 gradients
    outputs = sum(w.ns * w.nr * w.nt * 4 + 80 * w.nx * w.nz + 8 for w in jobs)
    arena = int((free - outputs) * 0.85) // 256 * 256
    eng = E.Engine(arena)
    grad_budget = arena // 16
    total_fwd = sum(cells(w) for w in jobs)

    clocks = Clocks(0)
    clocks.start()
    if profile:
        kernel_profile(True, every=8)
    # phase A: observed data of the true models (all shots of a job in one group when it fits)
    tickets = [eng.submit_model(grid_of(w), w.pz, s["a"], s["b"], s["src"], s["wav"], s["rec"],
                                work_budget=min(grad_budget, 1 << 62)) for w, s in zip(jobs, staged)]
    t_model, l_model, res = _drain(eng, tickets)
    data = [res[t].traces for t in tickets]
    # phase B: misfit and gradient of every job at the background model
    tickets = [eng.submit_gradient(grid_of(w), w.pz, s["zero"], s["zero"], s["src"], s["wav"], s["rec"], dd,
                                   work_budget=grad_budget) for w, s, dd in zip(jobs, staged, data)]
    t_grad, l_grad, res = _drain(eng, tickets)
    clk = clocks.stop()
    prof = kernel_profile(False) if profile else None
    finite = all(bool(torch.isfinite(res[t].grads).all()) for t in tickets[:8])
    eng.close()
    del eng, res
    torch.cuda.empty_cache()

    value = (total_fwd + 2 * total_fwd) / (t_model + t_grad) / 1e9
    plain = plain_per_shot_batch(jobs, staged, data, dev)
    out = {
        "value": round(value, 3), "unit": "Gcell-updates/s", "seconds": round(t_model + t_grad, 2),
        "jobs": njobs, "sample": f"the first {njobs} of batch_jobs({total}, seed 0)" if njobs < total else None,
        "sizes": "square 128^2..1024^2 (+40-cell sponge), 500-4000 steps, 1-32 shots, 8th order",
        "arena_gb": round(arena / 2**30, 1), "gradient_budget_gb": round(grad_budget / 2**30, 2),
        "forward": {"value": round(total_fwd / t_model / 1e9, 3), "seconds": round(t_model, 2),
                    "launches": l_model},
        "gradient": {"value": round(2 * total_fwd / t_grad / 1e9, 3), "seconds": round(t_grad, 2),
                     "gradients_per_s": round(njobs / t_grad, 3), "launches": l_grad, "finite": finite},
        "plain_per_shot": plain,
        "speedup_vs_plain": round(value / plain["value"], 2) if plain["value"] else None,
        "gpu_launches": l_model + l_grad, "clocks": clk,
    }
    if prof:
        out["profile"] = prof
    return out


def bench_batch(args, Clocks):
    r = run_batch(args.jobs, Clocks, profile=args.profile)
    out = {
        "metric": METRIC, "value": r["value"], "unit": "Gcell-updates/s", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": round(1e3 * r["seconds"], 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch-{args.jobs}-uneven", "jobs": args.jobs, "sizes": r["sizes"],
                   "arena_gb": r["arena_gb"], "gradient_budget_gb": r["gradient_budget_gb"],
                   "l2": "working set larger than L2"},
        **{k: r[k] for k in ("forward", "gradient", "plain_per_shot", "speedup_vs_plain", "gpu_launches", "clocks")},
    }
    if "profile" in r:
        out["profile"] = r["profile"]
    print(json.dumps(out), flush=True)


def plain_per_shot_batch(jobs, staged, data, dev, sample=16):
    """The plain per-shot GPU path on a seeded sample of the jobs: for the first `sample` jobs,
    shot 0 alone through fwi_model and fwi_gradient (one call each, workspace for one shot)."""
    upd, t = 0, 0.0
    for w, s, dd in list(zip(jobs, staged, data))[:sample]:
        g = grid_of(w)
        src = s["src"][:1]
        wm = F.workspace(g, 1, w.nr, F.OP_MODEL, 1 << 62)
        wg = F.workspace(g, 1, w.nr, F.OP_GRADIENT, 1 << 36)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.fwi_model(g, w.pz, s["a"], s["b"], src, s["wav"], s["rec"], work=wm, check=False)
        F.fwi_gradient(g, w.pz, s["zero"], s["zero"], src, s["wav"], s["rec"], dd[:1], work=wg, check=False)
        torch.cuda.synchronize()
        t += time.perf_counter() - t0
        upd += 3 * cells(w) // w.ns
        del wm, wg
    return {"value": round(upd / t / 1e9, 3), "unit": "Gcell-updates/s",
            "sample": f"shot 0 of the first {sample} jobs, model + gradient, one call each"}


# ------------------------------------------------------------------------------ serving

LIGHT = dict(side=(128, 256), steps=(500, 1000), shots=(1, 4))


def serve_requests(count, seed, **job_kw):
    """`count` requests, kinds uniform over forward / Born / gradient, sizes from
    inputs.batch_job(**job_kw)."""
    rng = np.random.default_rng(seed)
    kw = job_kw
    reqs = []
    for k in range(count):
        w = I.batch_job(np.random.SeedSequence([seed, 7, k]), **kw)
        kind = int(rng.integers(0, 3))
        r = S.Request(kind, w)
        if kind == E.JOB_BORN:
            r.dxi = (w.xi_a * np.float32(0.5), w.xi_b * np.float32(0.5))
            w.xi_a, w.xi_b = w.background()
        if kind == E.JOB_GRADIENT:
            r.data = I.random_like((w.ns, w.nr, w.nt), 10_000 + k, 1e3)
        reqs.append(r)
    return reqs


def serve_plain(requests, arrivals):
    """The same stream served one request at a time through the single-job calls."""
    n = len(requests)
    staged = [S.stage(r) for r in requests]
    done = np.zeros(n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, r in enumerate(requests):
        now = time.perf_counter() - t0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        w, st = r.workload, staged[k]
        g = grid_of(w)
        dv = lambda t: t.to("cuda", non_blocking=True)
        a, b, src, wav, rec = dv(st["a"]), dv(st["b"]), dv(st["src"]), dv(st["wav"]), dv(st["rec"])
        if r.kind == E.JOB_MODEL:
            F.fwi_model(g, w.pz, a, b, src, wav, rec, check=False)
        elif r.kind == E.JOB_BORN:
            F.fwi_born(g, w.pz, a, b, dv(st["da"]), dv(st["db"]), src, wav, rec, check=False)
        else:
            F.fwi_gradient(g, w.pz, a, b, src, wav, rec, dv(st["data"]), check=False)
        torch.cuda.synchronize()
        done[k] = time.perf_counter() - t0
    lat = done - arrivals[:n]
    upd = sum(PASSES[r.kind] * cells(r.workload) for r in requests)
    return {"req_per_s": round(n / done[-1], 2), "gcell_per_s": round(upd / done[-1] / 1e9, 3),
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2)}


def run_serve(requests, rate, sizes, Clocks, profile=False):
    """A seeded Poisson stream of `requests` mixed forward / Born / gradient requests at `rate`
    per second through the continuous-batching loop (sizes 'light' or 'batch'); the light stream
    is also served one request at a time through the single-job calls.  Returns a dict."""
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    kw = LIGHT if sizes == "light" else {}
    reqs = serve_requests(requests, seed=1, **kw)
    arrivals = I.poisson_arrivals(len(reqs), rate, seed=2)
    free, _ = torch.cuda.mem_get_info(dev)
    arena = int(free * 0.6) // 256 * 256
    # the engine: warm-up on the first few requests, then the timed stream
    S.serve(reqs[:4], np.zeros(4), arena)
    clocks = Clocks(0)
    clocks.start()
    if profile:
        kernel_profile(True, every=8)
    stats, _ = S.serve(reqs, arrivals, arena)
    prof = kernel_profile(False) if profile else None
    clk = clocks.stop()
    plain = serve_plain(reqs, arrivals) if sizes == "light" else None
    upd = sum(PASSES[r.kind] * cells(r.workload) for r in reqs)
    out = {"requests": len(reqs), "rate_per_s": rate, "mix": "forward / Born / gradient, uniform",
           "sizes": ("square 128^2..256^2, 500-1000 steps, 1-4 shots" if sizes == "light" else
                     "square 128^2..1024^2, 500-4000 steps, 1-32 shots"),
           "arena_gb": round(arena / 2**30, 1),
           "gcell_per_s": round(upd / stats["wall_s"] / 1e9, 3),
           **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in stats.items()},
           "plain_one_at_a_time": plain, "clocks": clk}
    if plain:
        out["speedup_vs_plain"] = round(stats["req_per_s"] / plain["req_per_s"], 2)
    if prof:
        out["profile"] = prof
    return out, reqs, arena


def bench_serve(args, Clocks):
    r, reqs, arena = run_serve(args.requests, args.rate, args.sizes, Clocks, profile=args.profile)
    stats = {k: r[k] for k in ("requests", "wall_s", "req_per_s", "p50_ms", "p99_ms", "mean_queue_ms", "launches",
                                "max_running")}
    kw = LIGHT if args.sizes == "light" else {}
    out = {
        "metric": METRIC, "value": r["gcell_per_s"], "unit": "Gcell-updates/s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": round(1e3 * stats["wall_s"], 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve-{args.sizes}-poisson{args.rate:g}", "requests": len(reqs),
                   "rate_per_s": args.rate, "mix": r["mix"], "sizes": r["sizes"], "arena_gb": r["arena_gb"]},
        "serving": stats,
        "plain_one_at_a_time": r["plain_one_at_a_time"],
        "gpu_launches": stats["launches"], "clocks": r["clocks"],
    }
    if args.capacity_run > 0:
        # a second stream at 80 % of the throughput the first one reached
        rate = 0.8 * stats["req_per_s"]
        reqs2 = serve_requests(args.capacity_run, seed=3, **kw)
        arr2 = I.poisson_arrivals(len(reqs2), rate, seed=4)
        st2, _ = S.serve(reqs2, arr2, arena)
        out["at_80pct_capacity"] = {"rate_per_s": round(rate, 3),
                                    **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in st2.items()}}
    if "profile" in r:
        out["profile"] = r["profile"]
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------- differentiation

def bench_differentiation(args, Clocks):
    """One FWI gradient through torch.autograd on the 1201 x 1201 smooth-background workload
    (6000 steps, 16 shots): forward modelling, a torch misfit, and the backward pass (adjoint
    with wavefield checkpoints every 200 steps and segment recomputation)."""
    from . import autograd as AG
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w, (a_bg, b_bg) = I.config_smooth()
    g = grid_of(w)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    src, rec, wav = d(w.src_xy), d(w.rec_xy), d(w.wavelet)
    data = F.fwi_model(g, w.pz, d(w.xi_a), d(w.xi_b), src, wav, rec)
    F.fwi_set_checkpoint(200)
    launches = [0]

    def step():
        a0 = d(a_bg).requires_grad_()
        b0 = d(b_bg).requires_grad_()
        tr = AG.model(a0, b0, g, w.pz, src, wav, rec)
        launches[0] += F.launch_count()
        J = 0.5 * ((tr.double() - data.double()) ** 2).sum()
        J.backward()
        launches[0] += AG.FwiFunction.last_backward_launches
        return J, a0.grad, b0.grad

    try:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        launches[0] = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            J, ga, gb = step()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
    finally:
        F.fwi_set_checkpoint(0)
    ms = e0.elapsed_time(e1) / args.steps
    upd = 3 * cells(w)          # forward + (forward history + adjoint); recomputation not counted
    out = {
        "metric": METRIC, "value": round(upd / (ms / 1e3) / 1e9, 3), "unit": "Gcell-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "gradients_per_s": round(1e3 / ms, 4),
        "config": {"workload": "smooth-1201x1201-o8 (autograd, checkpoints every 200 steps)",
                   "grid": "1201x1201 + 40-cell sponge = 1281x1281", "nt": w.nt, "shots": w.ns, "receivers": w.nr,
                   "step": "traces = FwiFunction(xi_a, xi_b); J = 1/2 |traces - data|^2 (torch); J.backward()",
                   "passes": "forward 1 + backward (forward with checkpoints 1, recompute 1, adjoint 1)"},
        "misfit": float(J.item()), "gradient_finite": bool(torch.isfinite(ga).all() and torch.isfinite(gb).all()),
        "gpu_launches": launches[0] // max(args.steps, 1), "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------ error bowls

def bench_bowls(args, Clocks):
    """Error bowls of scatterer `args.case` (paper acquisition, 121 x 121 + 40-cell sponge,
    1400 steps, 10 shots, 100 receivers, 5 Hz) in all five parameterizations, 21 x 21 contrasts
    each: 2205 forward solves through the batching engine."""
    from . import bowls as B
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.case not in B.CASES:
        raise SystemExit("error bowls need a known-shape scatterer: --case i, ii, iv or v")
    if args.scheme in (1, 2):
        return bench_born_bowls(args, Clocks)
    w, g = B.scatterer(args.case)
    shape, which = B.CASES[args.case]
    amp = 0.2
    ranges = {"all": None, "short": (0.0, 90.0), "long": (135.0, 180.0)}[args.aperture]
    weights = None if ranges is None else B.aperture_weights(w.src_xy, w.rec_xy, I.centre_of(w.nx, w.nz, w.dx),
                                                             *ranges)
    data = F.fwi_model(grid_of(w), I.PZ_VP_RHO, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    dvp, drho = (amp, 0.0) if which == "vp" else (0.0, amp)
    grids = {}
    for pz in range(5):
        ta, tb = B.true_point(pz, dvp, drho)
        grids[pz] = (B.grid_around(ta, args.bowl_n), B.grid_around(tb, args.bowl_n))
    B.error_bowl(w, g, I.PZ_K_RHO, data, grids[I.PZ_K_RHO][0][:3], grids[I.PZ_K_RHO][1][:3])   # warm-up
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    shapes, launches = {}, 0
    for pz in range(5):
        J, l = B.error_bowl(w, g, pz, data, *grids[pz], weights=weights)
        launches += l
        shapes[["vp-rho", "Ip-rho", "vp-Ip", "K-rho", "1/K-1/rho"][pz]] = {
            k: (round(v, 4) if isinstance(v, float) else [round(x, 4) for x in v]) for k, v in B.bowl_shape(J, *grids[pz]).items()}
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    solves = 5 * args.bowl_n ** 2
    upd = solves * cells(w)
    out = {
        "metric": METRIC, "value": round(upd / wall / 1e9, 3), "unit": "Gcell-updates/s", "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": round(1e3 * wall, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"bowls-scatterer-{args.case}-aperture-{args.aperture}",
                   "scatterer": f"{shape}, {which} only, contrast {amp}",
                   "scattering_angles": "all" if ranges is None else f"{ranges[0]:g}-{ranges[1]:g} degrees",
                   "grid": "121x121 + 40-cell sponge, dx 10 m, 8th order, 1400 steps, 10 shots, 100 receivers, 5 Hz",
                   "bowl": f"{args.bowl_n}x{args.bowl_n} contrasts per parameterization, 5 parameterizations"},
        "solves_per_s": round(solves / wall, 2), "bowls": shapes, "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(out), flush=True)


def bench_born_bowls(args, Clocks):
    """Error bowls of scatterer `args.case` under Schemes I/II: the frequency-domain Born misfit
    (paper acquisition, 121 x 121 nodes at 5 m, 60 frequencies) over the same contrast grids as
    the time-domain bowls; observed data from the exact map."""
    from . import bowls as B
    from . import fborn as FBN
    if args.aperture != "all":
        raise SystemExit("the frequency-domain bowls use every scattering angle")
    shape, which = B.CASES[args.case]
    w = I.freq_paper(which=which, shape=shape)
    h = (w.nx - 1) / 2 * w.dx
    g = I.point(w.nx, w.nz) if shape == "point" else I.gaussian(w.nx, w.nz, w.dx, (h, h), 50.0)
    acq = FBN.acquisition(w)
    data = acq.model(I.PZ_VP_RHO, w.xi_a, w.xi_b, scheme=FBN.NONLINEAR)
    amp = 0.2
    dvp, drho = (amp, 0.0) if which == "vp" else (0.0, amp)
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    shapes = {}
    for pz in range(5):
        ta, tb = B.true_point(pz, dvp, drho)
        ga, gb = B.grid_around(ta, args.bowl_n), B.grid_around(tb, args.bowl_n)
        J = B.born_error_bowl(acq, g, pz, data, ga, gb, args.scheme)
        shapes[["vp-rho", "Ip-rho", "vp-Ip", "K-rho", "1/K-1/rho"][pz]] = {
            k: (round(v, 4) if isinstance(v, float) else [round(x, 4) for x in v])
            for k, v in B.bowl_shape(J, ga, gb).items()}
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    points = 5 * args.bowl_n ** 2
    out = {
        "metric": "Born W-terms/s (frequency x source x receiver x node products), Schemes I/II",
        "value": round(points * w.terms() / wall / 1e9, 3), "unit": "GW-terms/s", "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": round(1e3 * wall, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"born-bowls-scheme{args.scheme}-scatterer-{args.case}",
                   "scatterer": f"{shape}, {which} only, contrast {amp}",
                   "grid": "121x121 nodes, dx 5 m, 10 sources, 100 receivers, 60 frequencies",
                   "bowl": f"{args.bowl_n}x{args.bowl_n} contrasts per parameterization, 5 parameterizations"},
        "misfits_per_s": round(points / wall, 1), "bowls": shapes, "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# -------------------------------------------------------------------------------- inversion

def bench_invert(args, Clocks):
    """Steepest descent on scatterer `args.case` (known shape: the two contrasts are the
    unknowns) in all five parameterizations, from the homogeneous starting model; reports each
    misfit history (the convergence ranking).  --scheme 3 (default): time-domain modelling,
    the line search's trial models as batching-engine jobs; --scheme 1 or 2: the
    frequency-domain Born path under the linear (Scheme I) or exact (Scheme II) map, observed
    data from the exact map."""
    from . import bowls as B
    from . import invert as V
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    names = ["vp-rho", "Ip-rho", "vp-Ip", "K-rho", "1/K-1/rho"]
    known = args.case in B.CASES
    kind = "known-shape" if known else "unknown-shape"
    if args.scheme in (1, 2):
        from . import fborn as FBN
        if known:
            shape, which = B.CASES[args.case]
            w = I.freq_paper(which=which, shape=shape)
            g = (I.point(w.nx, w.nz) if shape == "point"
                 else I.gaussian(w.nx, w.nz, w.dx, ((w.nx - 1) / 2 * w.dx, (w.nz - 1) / 2 * w.dx), 50.0))
        else:
            w = I.freq_paper()
            gu = I.gaussian(w.nx, w.nz, w.dx, ((w.nx - 1) / 2 * w.dx, (w.nz - 1) / 2 * w.dx), 50.0)
            w.xi_a, w.xi_b = B.unknown_contrasts(gu, B.UNKNOWN[args.case])
            g = None
        acq = FBN.acquisition(w)
        data = acq.model(I.PZ_VP_RHO, w.xi_a, w.xi_b, scheme=FBN.NONLINEAR)
        make = lambda pz: V.BornInversion(acq, pz, data, args.scheme, shape=g)
        line_search = "8 trial steps a iteration (fwi_fborn_misfit)"
        label = f"invert-scheme{args.scheme}-scatterer-{args.case}-{kind}"
    else:
        if known:
            w, g = B.scatterer(args.case)
        else:
            w, g = B.unknown_scatterer(args.case), None
        data = F.fwi_model(grid_of(w), I.PZ_VP_RHO, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
        make = lambda pz: V.Inversion(w, pz, data, shape=g)
        line_search = "8 trial steps a iteration as engine jobs"
        label = f"invert-scatterer-{args.case}-{kind}"
    zero = lambda: torch.zeros((w.nz, w.nx), dtype=torch.float32, device=dev)
    m0 = (lambda: (0.0, 0.0)) if known else (lambda: (zero(), zero()))
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    res = {}
    for pz in range(5):
        inv = make(pz)
        m, hist = inv.run(m0(), iters=args.iters)
        inv.close()
        final = ([round(m[0], 5), round(m[1], 5)] if known else
                 [round(float(m[0].abs().max()), 5), round(float(m[1].abs().max()), 5)])
        res[names[pz]] = {("final" if known else "final_max_abs"): final,
                          "misfit": [float(f"{j:.5g}") for j in hist],
                          "reduction": float(f"{hist[-1] / hist[0]:.4g}")}
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    out = {
        "metric": METRIC, "value": round(wall, 2), "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": round(1e3 * wall, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": label, "iterations": args.iters, "line_search": line_search},
        "inversions": res, "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ frequency-domain Born (I/II)

FB_FLOPS_PER_TERM = 24      # three complex multiply-adds per (frequency, source, receiver, node)
FP32_LANES_PER_SM = 128


def measured_hbm_gbs():
    """(HBM copy bandwidth in GB/s, its source): MEASURED_PEAKS.json's hbm_gbs at the repository
    root, else the machine's fallback figure."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        if "hbm_gbs" in pk:
            return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback"


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak of the GPU at the given SM clock: SMs x 128 lanes x 2 flops x clock."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def bench_fborn(args, Clocks, cpu_sample=None):
    """Frequency-domain Born kernels of Schemes I/II on the paper's acquisition (121 x 121
    nodes at 5 m around x_0, 10 sources and 100 receivers on the 490 m circle, 60 frequencies
    0.25 - 15 Hz with the 5 Hz Ricker spectrum; observed data of the Gaussian vp scatterer,
    contrast 0.2, under the exact map).  One step: for each of the five parameterizations, the
    Scheme I misfit gradient at a seeded model (data contraction, misfit, gradient contraction)
    and the Hessian column at x_0 (whose centre is the reduced Hessian).  A term is one
    (frequency, source, receiver, node) product of W; a gradient takes two passes over them.
    cpu_sample(w), when given, times the CPU baseline."""
    from . import fborn as FBN
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = I.freq_paper()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    acq = FBN.acquisition(w)
    torch.cuda.synchronize()
    tables_ms = 1e3 * (time.perf_counter() - t0)
    q = acq.model(I.PZ_VP_RHO, w.xi_a, w.xi_b, scheme=FBN.NONLINEAR)
    models = [(torch.from_numpy(I.random_like((w.nz, w.nx), 40 + pz, 0.05)).to(dev),
               torch.from_numpy(I.random_like((w.nz, w.nx), 50 + pz, 0.05)).to(dev)) for pz in range(5)]
    J = torch.empty((5, 1), dtype=torch.float64, device=dev)
    G = torch.empty((5, 2, w.nz, w.nx), dtype=torch.float64, device=dev)
    H = torch.empty((5, 2, 2, w.nz, w.nx), dtype=torch.float64, device=dev)
    c = w.nx // 2

    def step():
        # gradient and Hessian column in one pass over the tables (fwi_fborn_gradient_hessian)
        for pz in range(5):
            acq.gradient_hessian(pz, *models[pz], q, c, c, scheme=FBN.LINEAR, misfit=J[pz], grad=G[pz], H=H[pz])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    kernel_profile(True)
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = kernel_profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    terms = w.terms()
    passes = 2 * 5
    # end to end through the public API: host contrasts and observed data in, misfit, gradient
    # and Hessian column out to host memory, every step
    host_models = [(m[0].cpu().numpy(), m[1].cpu().numpy()) for m in models]
    q_host = q.cpu().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for pz in range(5):
            Jh, Gh, Hh = acq.gradient_hessian(pz, *host_models[pz], q_host, c, c, scheme=FBN.LINEAR)
            Jh.cpu(), Gh.cpu(), Hh.cpu()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = 5 * (2 * w.nx * w.nz * 4 + q_host.nbytes)
    d2h = 5 * (8 + 2 * w.nx * w.nz * 8 + 4 * w.nx * w.nz * 8)
    # rooflines: the tensor-core data contraction is bound by streaming the tables from HBM
    # (every table value of every point read once, plus the chunk partials written); the
    # gradient and the Hessian column by the FP32 pipe (24 algorithmic flops per term)
    kern = prof["kernels"]
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    fp32_peak = fp32_peak_tflops(sm_mhz)
    hbm_peak, hbm_src = measured_hbm_gbs()
    P, N = w.src_xy.shape[0] + w.rec_xy.shape[0], w.nx * w.nz
    nchunk = (N + 255) // 256
    table_bytes = 16 * w.nf * P * N + 8 * nchunk * w.nf * w.src_xy.shape[0] * w.rec_xy.shape[0]
    flops = FB_FLOPS_PER_TERM * terms

    def traffic(k):
        """DRAM bytes per launch from the committed ncu capture (profiles/traffic_fborn.json);
        None when the kernels changed since it was taken."""
        import hashlib
        import json
        import os
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        path = os.path.join(root, "profiles", "traffic_fborn.json")
        if not os.path.exists(path):
            return None
        t = json.load(open(path))
        src = open(os.path.join(root, "paper_1804_01184_gb300", "csrc", "fwi_fborn.inc"), "rb").read()
        short = k.split("::")[-1].split("<")[0]
        if t.get("kernel_source_sha256") != hashlib.sha256(src).hexdigest() or short not in t.get("kernels", {}):
            return None
        return t["kernels"][short]["dram_bytes_per_launch"]

    def roof(k):
        per_launch_ms = kern[k]["ms"] / kern[k]["launches"]
        if "model_tc" in k:
            a = table_bytes / (per_launch_ms / 1e3) / 1e9
            return {"kernel": k, "bound": "hbm", "achieved": round(a, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(a / hbm_peak, 4), "traffic": traffic(k), "bytes_per_launch": table_bytes,
                    "avg_launch_us": round(1e3 * per_launch_ms, 2), "peak_source": hbm_src}
        # the Hessian column's Gram sums: 9 complex multiply-adds (72 flops) per (frequency, point,
        # node); the gradient pass that also forms them (k_fb_grad<., true>) does both
        hess_flops = 72 * w.nf * P * N
        fl = hess_flops if "hess" in k else flops + (hess_flops if "true" in k else 0)
        a = fl / (per_launch_ms / 1e3) / 1e12
        return {"kernel": k, "bound": "alu", "achieved": round(a, 2), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(a / fp32_peak, 4), "traffic": traffic(k), "flops_per_launch": fl,
                "avg_launch_us": round(1e3 * per_launch_ms, 2),
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 flops x max SM clock"}

    name = max(kern, key=lambda k: kern[k]["ms"])
    roofline = roof(name)
    rooflines = {k: roof(k) for k in kern if any(t in k for t in ("model_tc", "k_fb_grad<", "k_fb_hess"))
                 and "sum" not in k}
    cpu = cpu_sample(w) if (cpu_sample and not args.no_cpu) else None
    # diffraction patterns (Sec. "Diffraction-pattern Analysis"): energy scattered by a unit
    # point contrast of each parameter at x_0, relative to its maximum, by scattering angle
    from . import patterns as PT
    ang = PT.scattering_angles(w.src_xy, w.rec_xy, (0.0, 0.0))
    pnames = [("vp", "rho"), ("Ip", "rho"), ("vp", "Ip"), ("K", "rho"), ("1/K", "1/rho")]
    patterns = {}
    for pz in range(5):
        for k in range(2):
            patterns[f"{pnames[pz][k]} in {['vp-rho', 'Ip-rho', 'vp-Ip', 'K-rho', '1/K-1/rho'][pz]}"] = \
                PT.pattern_summary(PT.diffraction_pattern(acq, pz, k, c, c), ang)
    # the point-scatterer analysis (Sec. "Point-scatterer Analysis"): the reduced Hessian at x_0
    # of each parameterization -- condition number, cross-parameter ratio, long-axis angle
    names = ["vp-rho", "Ip-rho", "vp-Ip", "K-rho", "1/K-1/rho"]
    reduced = {}
    for pz in range(5):
        Hr = H[pz, :, :, c, c].cpu().numpy()
        Hs = 0.5 * (Hr + Hr.T)
        lam, vec = np.linalg.eigh(Hs)
        reduced[names[pz]] = {"condition": float(f"{lam[1] / lam[0]:.4g}"),
                              "cross_ratio": float(f"{Hs[0, 1] / np.sqrt(Hs[0, 0] * Hs[1, 1]):.3g}"),
                              "long_axis_deg": round(float(np.degrees(np.arctan2(vec[1, 0], vec[0, 0])) % 180.0), 1)}
    out = {
        "metric": "Born W-terms/s (frequency x source x receiver x node products), Schemes I/II",
        "value": round(passes * terms / (ms / 1e3) / 1e9, 3), "unit": "GW-terms/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "freq-born-paper-121x121", "grid": "121x121 nodes, dx 5 m, centred on x_0",
                   "acquisition": "10 sources, 100 receivers, 490 m circle", "frequencies": "60 (0.25-15 Hz)",
                   "step": "5 x (Scheme I gradient + Hessian column at x_0, one table pass for both)",
                   "l2": "Green tables 1.55 GB, larger than L2", "tables_ms": round(tables_ms, 1)},
        "roofline": roofline, "kernel_rooflines": rooflines,
        "kernels": kern, "gpu_launches": sum(v["launches"] for v in kern.values()) // max(args.steps, 1),
        "clocks": clk,
        "e2e": {"value": round(passes * terms / e2e_s / 1e9, 3), "unit": "GW-terms/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu,
        "reduced_hessian_x0": reduced,
        "diffraction_patterns": patterns,
    }
    print(json.dumps(out), flush=True)

