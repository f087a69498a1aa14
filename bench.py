#!/usr/bin/env python
"""Benchmark of the Scheme III hot path (arXiv:1804.01184) on GB300.

One step = one pass of the whole hot path over one batch of the Gaussian-scatterer workload
(601 x 601 physical nodes + 40-cell sponge = 681 x 681, dx 5 m, 8th order, dt 0.5 ms, 3000
steps, 64 sources / 256 receivers on a 1200 m circle, Gaussian sigma 20 m, contrast swept
over [-0.5, 0.5] in vp and in rho, one value per step):
  1. fwi_model    : observed data of the true model                     (model build, forward)
  2. fwi_gradient : misfit and gradient at the background for all five   (forward + snapshots,
                    parameterizations                                      residual, adjoint, chain rule)
  3. fwi_born     : Born traces of the true contrast around the background
Metric: algorithmic cell-updates per second (computational cells incl. sponge x steps x
shots x propagation passes: model 1, gradient 2 (forward + adjoint), Born 1; recomputed
forward steps are not counted) and FWI gradients per second.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; every rank solves its own problems (different
contrasts), so there is no collective on the data path ("weak" scaling).

Two more workloads run through the batching engine (one JSON line each, 1 GPU):
  --workload batch : 256 uneven jobs (square grids 128^2..1024^2, 500-4000 steps, 1-32 shots,
                     point or Gaussian scatterers): their forward models (the observed data),
                     then their misfit gradients at the background, each phase as one engine
                     run; against the plain per-shot GPU path on a seeded sample of the jobs.
  --workload serve : a seeded Poisson stream of mixed forward / Born / gradient requests with
                     continuous batching; throughput and p50/p99 latency, against serving the
                     same stream one request at a time through the single-job calls.
  --workload bowls : error bowls of a known-shape scatterer in all five parameterizations
                     (2205 forward solves through the batching engine).
  --workload invert : steepest-descent inversions of a known-shape scatterer in all five
                     parameterizations (line searches as engine jobs); misfit histories.
  --workload differentiation : one FWI gradient through torch.autograd on the 1201 x 1201,
                     6000-step, 16-shot smooth-background workload with checkpoints every 200
                     steps (per step: forward, torch misfit, backward).
  --workload fborn : the frequency-domain Born path of Schemes I/II on the paper's acquisition
                     (per step, for each parameterization: a Scheme I gradient and the Hessian
                     column at x_0); Born W-terms per second.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s & FWI gradients/s vs plain per-shot GPU; p50/p99 solve latency"
UNIT = "Gcell-updates/s"

# Algorithmic HBM bytes per computational cell and shot for one launch of each time-step kernel
# (FP32 fields, each read or written once), and model bytes per cell counted once per launch
# (the model arrays are shared by every shot of the launch).
KERNEL_BYTES = {
    "k_fwd_warp": 24,    # p^n, vx, vz read; p^{n+1}, vx, vz written
    "k_adj_warp": 52,    # pbar, vbar read+written (24), p^n snapshot (4), g_K, g_bx, g_bz accumulated (24)
    "k_born_warp": 48,   # background and scattered p, vx, vz read and written
}
MODEL_BYTES = {"k_fwd_warp": 12, "k_adj_warp": 12, "k_born_warp": 24}


def short_name(launch_name):
    """'(fwi::k_fwd_warp<4, 1>)' -> 'k_fwd_warp'"""
    return launch_name.split("::")[-1].split("<")[0].strip("()")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("fwi_warp.cuh", "fwi_stream.cuh", "fwi_kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1804_01184_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(kernel, shots):
    """DRAM bytes (read + write) per launch from the committed ncu capture, scaled to `shots`
    shots per launch; None when the kernels changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    t = json.load(open(path))
    if t.get("kernel_source_sha256") != kernel_source_hash() or kernel not in t.get("kernels", {}):
        return None
    k = t["kernels"][kernel]
    return int(k["dram_bytes_per_launch"] * shots / k["shots_per_launch"])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nt", type=int, default=3000)
    ap.add_argument("--shots", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-engine", action="store_true",
                    help="skip the batching and serving measurements that follow the main one")
    ap.add_argument("--engine-jobs", type=int, default=32,
                    help="batching measurement: the first N of the 256 uneven jobs")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="serving measurement: requests of the light Poisson stream")
    ap.add_argument("--profile-every", type=int, default=8,
                    help="time one launch in N of each kernel with CUDA events inside the timed region")
    ap.add_argument("--tile", type=int, default=0,
                    help="fixed strip height of the streaming kernels (0: tuned online; profiling uses a fixed one)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="gradient workspace budget (0: 80%% of free device memory)")
    ap.add_argument("--workload", default="gaussian",
                    choices=["gaussian", "batch", "serve", "differentiation", "bowls", "invert", "fborn"])
    ap.add_argument("--iters", type=int, default=15, help="invert: iterations")
    ap.add_argument("--scheme", type=int, default=3, choices=[1, 2, 3],
                    help="invert / bowls: 3 time-domain modelling (Scheme III); 1, 2 frequency-domain Born "
                         "(Schemes I, II)")
    ap.add_argument("--case", default="ii", choices=["i", "ii", "iii", "iv", "v", "vi", "vii"],
                    help="bowls / invert: scatterer (iii, vi, vii: unknown shape, invert only)")
    ap.add_argument("--bowl-n", type=int, default=21, help="bowls: contrasts per axis")
    ap.add_argument("--aperture", default="all", choices=["all", "short", "long"],
                    help="bowls: scattering angles used (short: 0-90, long: 135-180 degrees)")
    ap.add_argument("--jobs", type=int, default=256, help="batch: number of jobs")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--profile", action="store_true", help="batch/serve: per-kernel device time")
    ap.add_argument("--capacity-run", type=int, default=0,
                    help="serve: requests of a second stream at 80%% of the first stream's throughput")
    ap.add_argument("--sizes", default="light", choices=["light", "batch"],
                    help="serve: request sizes (light: 128-256^2, 500-1000 steps, 1-4 shots; "
                         "batch: the batch workload's distribution)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def contrast_of(k, rank):
    """Step k of rank r: amplitude from the sweep {-0.5, ..., 0.5} \\ {0}, vp then rho."""
    amps = [a / 10 for a in range(-5, 6) if a != 0]
    idx = (k + 7 * rank) % (2 * len(amps))
    return amps[idx % len(amps)], ("vp" if idx < len(amps) else "rho")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------------------- oracle arm

def cpu_sample(nt_sample=300, shots=(0,)):
    """The FP64 oracle on a bounded sample of the workload: the same three calls for the
    listed shots over the first nt_sample steps.  Returns (Gcell-updates/s, seconds, cores)."""
    import numpy as np

    import oracle
    from paper_1804_01184_gb300 import inputs as I
    amp, which = contrast_of(0, 0)
    w = I.config_gaussian(amp, which, nt=nt_sample)
    w = w.subset(list(shots))
    g = oracle.make_grid(**w.grid_kwargs())
    a0, b0 = w.background()
    t0 = time.perf_counter()
    data = oracle.model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    oracle.gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data.astype(np.float32))
    oracle.born(g, w.pz, a0, b0, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    dt = time.perf_counter() - t0
    cells = w.Nx * w.Nz * w.nt * w.ns * 4
    return cells / dt / 1e9, dt, cells

def fborn_cpu_sample(w, nf=2):
    """The FP64 oracle's Scheme I gradient on the first nf frequencies of the workload (full
    grid and acquisition), scaled to W-terms per second (two passes)."""
    import numpy as np

    import oracle.fborn as OF
    fg = OF.FGrid(**w.fgrid_kwargs())
    fr, sp = w.freqs[:nf], w.spectrum[:nf]
    q = OF.model(fg, fr, sp, w.src_xy, w.rec_xy, 0, w.xi_a, w.xi_b, OF.NONLINEAR)
    a0 = np.zeros_like(w.xi_a, dtype=np.float64)
    t0 = time.perf_counter()
    OF.gradient(fg, fr, sp, w.src_xy, w.rec_xy, 0, a0, a0, q, OF.LINEAR)
    dt = time.perf_counter() - t0
    terms = nf * w.ns * w.nr * w.nx * w.nz
    return {"value": round(2 * terms / dt / 1e9, 4), "unit": "GW-terms/s", "cores": 1,
            "kind": "oracle", "sample": f"Scheme I gradient (vp-rho), {nf} of {w.nf} frequencies, full grid and "
                                        f"acquisition (numpy FP64, one thread, {dt:.1f} s)"}


def run_reference(args, rank):
    if rank != 0:
        return
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    nt_s = 200
    for _ in range(args.warmup):
        cpu_sample(nt_s)
    times, cells = [], 0
    for _ in range(args.steps):
        _, dt, cells = cpu_sample(nt_s)
        times.append(dt)
    total = sum(times)
    value = cells * args.steps / total / 1e9
    sample = f"1 of 64 shots, first {nt_s} of 3000 steps, full 681x681 grid: model + gradient + born (FP64 C oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gaussian-601x601-o8 (bounded oracle sample)", "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------ GPU arm

def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload != "gaussian":
        from paper_1804_01184_gb300 import workloads
        {"batch": workloads.bench_batch, "serve": workloads.bench_serve,
         "differentiation": workloads.bench_differentiation, "bowls": workloads.bench_bowls,
         "invert": workloads.bench_invert,
         "fborn": lambda a, c: workloads.bench_fborn(a, c, fborn_cpu_sample)}[args.workload](args, Clocks)
        return
    import numpy as np
    import torch

    from paper_1804_01184_gb300 import fwi
    from paper_1804_01184_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    fwi.lib()
    if args.tile:
        fwi.fwi_set_tile(args.tile, 0)

    nt, ns = args.nt, args.shots
    w0 = I.config_gaussian(0.3, "vp", nt=nt, ns=ns)
    g = fwi.make_grid(**w0.grid_kwargs())
    nr = w0.nr
    src = torch.from_numpy(w0.src_xy).to(dev)
    rec = torch.from_numpy(w0.rec_xy).to(dev)
    wav = torch.from_numpy(w0.wavelet).to(dev)
    zero = torch.zeros((w0.nz, w0.nx), dtype=torch.float32, device=dev)

    # the contrasts of every step, resident in HBM before the timed region
    nsteps = args.warmup + args.steps
    models = []
    for k in range(nsteps):
        amp, which = contrast_of(k, rank)
        wk = I.config_gaussian(amp, which, nt=nt, ns=ns)
        models.append((torch.from_numpy(wk.xi_a).to(dev), torch.from_numpy(wk.xi_b).to(dev)))

    ws_model = fwi.workspace(g, ns, nr, fwi.OP_MODEL)
    ws_born = fwi.workspace(g, ns, nr, fwi.OP_BORN)
    data = torch.empty((ns, nr, nt), dtype=torch.float32, device=dev)
    dtr = torch.empty_like(data)
    grads = torch.empty((5, 2, w0.nz, w0.nx), dtype=torch.float64, device=dev)
    misfit = torch.empty((), dtype=torch.float64, device=dev)
    ws_grad = fwi.workspace(g, ns, nr, fwi.OP_GRADIENT,
                            int(args.budget_gb * 2**30) if args.budget_gb > 0 else None)
    stream = torch.cuda.current_stream(dev)
    launches = [0]

    def step(k, check=False):
        xa, xb = models[k]
        fwi.fwi_model(g, w0.pz, xa, xb, src, wav, rec, traces=data, work=ws_model, check=check)
        launches[0] += fwi.launch_count()
        fwi.fwi_gradient(g, w0.pz, zero, zero, src, wav, rec, data, misfit=misfit, grads=grads,
                         work=ws_grad, check=check)
        launches[0] += fwi.launch_count()
        fwi.fwi_born(g, w0.pz, zero, zero, xa, xb, src, wav, rec, dtraces=dtr, work=ws_born, check=check)
        launches[0] += fwi.launch_count()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for k in range(args.warmup):
        step(k, check=(k == 0))
    torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    clocks.start()
    fwi.lib().fwi_profile(max(1, args.profile_every))
    launches[0] = 0
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup, nsteps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    fwi.lib().fwi_profile(0)
    clk = clocks.stop()
    buf = __import__("ctypes").create_string_buffer(1 << 16)
    fwi.lib().fwi_profile_report(buf, len(buf))
    prof = {}
    for line in buf.value.decode().splitlines():
        name, seen, cnt, tot = line.rsplit(" ", 3)
        # all launches of the kernel, and its device time estimated from the timed ones
        prof[name] = (int(seen), float(tot) / int(cnt) * int(seen), int(cnt))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()

    cells = w0.Nx * w0.Nz
    upd_per_step = cells * nt * ns * 4            # model 1 + gradient 2 + Born 1
    value = upd_per_step * args.steps * world / (ms / 1e3) / 1e9
    grads_per_s = args.steps * world / (ms / 1e3)

    # roofline of the dominant kernel (largest share of device time in the timed region)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    total_dev = sum(v[1] for v in prof.values()) or 1.0
    kernels = {}
    for name, (cnt, tot, timed) in prof.items():
        kernels[name.replace("fwi::", "").replace("(", "").replace(")", "").replace(", ", ",")] = {
            "launches": cnt, "timed_launches": timed, "ms": round(tot, 3), "share": round(tot / total_dev, 4)}
    # shot-steps each time-step kernel performs per bench step: the forward runs in fwi_model
    # and in fwi_gradient, the adjoint in fwi_gradient, Born in fwi_born
    shot_steps = {"k_fwd_warp": 2 * ns * nt, "k_adj_warp": ns * nt, "k_born_warp": ns * nt}
    roof = None
    dom = max(((n, v) for n, v in prof.items() if short_name(n) in KERNEL_BYTES), key=lambda kv: kv[1][1],
              default=None)
    if dom:
        name, (cnt, tot, _) = dom
        short = short_name(name)
        shots = shot_steps[short] * args.steps / cnt          # average shots per launch
        bytes_per_launch = cells * (KERNEL_BYTES[short] * shots + MODEL_BYTES[short])
        avg_s = tot / cnt / 1e3
        achieved = bytes_per_launch / avg_s / 1e9
        roof = {"kernel": short, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": measured_traffic(short, shots),
                "bytes_per_launch": int(bytes_per_launch), "shots_per_launch": round(shots, 2),
                "avg_launch_us": round(avg_s * 1e6, 2),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "gradients_per_s": round(grads_per_s, 4),
        "config": {"workload": "gaussian-601x601-o8", "grid": "601x601 + 40-cell sponge = 681x681", "dx_m": 5.0,
                   "order": 8, "nt": nt, "shots": ns, "receivers": nr,
                   "step": "fwi_model(true) + fwi_gradient(background, 5 parameterizations) + fwi_born(background)",
                   "l2": "working set larger than L2 (wavefield state alone %d MB)" % (3 * ns * cells * 4 >> 20),
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "gradient_plan": "workspace %.1f GB" % (ws_grad.numel() / 2**30)},
        "roofline": roof, "kernels": kernels, "gpu_launches": launches[0] * world, "clocks": clk,
    }

    if rank == 0 and not args.no_plain:
        out["plain_per_shot"] = plain_per_shot(fwi, I, g, w0, dev, nt)
    if not args.no_e2e:
        out["e2e"] = end_to_end(fwi, I, g, w0, dev, nt, ns, args, rank, world, (ws_model, ws_grad, ws_born))
    if rank == 0 and world == 1 and not args.no_engine:
        # the batching engine and the serving loop (the workloads' own sizes; each with its own
        # clock record): the main workspaces go first
        del ws_model, ws_grad, ws_born
        torch.cuda.empty_cache()
        from paper_1804_01184_gb300 import workloads
        out["batching"] = workloads.run_batch(args.engine_jobs, Clocks)
        torch.cuda.empty_cache()
        out["serving"] = workloads.run_serve(args.serve_requests, 200.0, "light", Clocks)[0]
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        v, dt, _ = cpu_sample(300)
        out["cpu_baseline"] = {"value": round(v, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "1 of 64 shots, first 300 of 3000 steps, full 681x681 grid: model + "
                                         "gradient + born (FP64 C oracle, %.1f s)" % dt}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def plain_per_shot(fwi, I, g, w0, dev, nt, shots=4):
    """The same step for a few shots, one shot at a time (workspaces sized for one shot):
    the plain per-shot GPU path, no batching, no graphs."""
    import torch
    sub = w0.subset(range(shots))
    src = torch.from_numpy(sub.src_xy).to(dev)
    rec = torch.from_numpy(w0.rec_xy).to(dev)
    wav = torch.from_numpy(w0.wavelet).to(dev)
    xa, xb = torch.from_numpy(w0.xi_a).to(dev), torch.from_numpy(w0.xi_b).to(dev)
    zero = torch.zeros_like(xa)
    nr = w0.nr
    wm = fwi.workspace(g, 1, nr, fwi.OP_MODEL, fwi.fwi_workspace_bytes(g, 1, nr, fwi.OP_MODEL, 0))
    wb = fwi.workspace(g, 1, nr, fwi.OP_BORN, fwi.fwi_workspace_bytes(g, 1, nr, fwi.OP_BORN, 0))
    wg = fwi.workspace(g, 1, nr, fwi.OP_GRADIENT, fwi.fwi_workspace_bytes(g, 1, nr, fwi.OP_GRADIENT, 1 << 62))
    data = torch.empty((1, nr, nt), dtype=torch.float32, device=dev)
    dtr = torch.empty_like(data)
    grads = torch.empty((5, 2, w0.nz, w0.nx), dtype=torch.float64, device=dev)
    misfit = torch.empty((), dtype=torch.float64, device=dev)

    def one(s):
        fwi.fwi_model(g, w0.pz, xa, xb, src[s:s + 1], wav, rec, traces=data, work=wm, check=False)
        fwi.fwi_gradient(g, w0.pz, zero, zero, src[s:s + 1], wav, rec, data, misfit=misfit, grads=grads, work=wg,
                         check=False)
        fwi.fwi_born(g, w0.pz, zero, zero, xa, xb, src[s:s + 1], wav, rec, dtraces=dtr, work=wb, check=False)

    one(0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for s in range(shots):
        one(s)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    upd = w0.Nx * w0.Nz * nt * shots * 4
    return {"value": round(upd / dt / 1e9, 3), "unit": UNIT, "shots": shots,
            "ms_per_shot": round(1e3 * dt / shots, 2)}


def end_to_end(fwi, I, g, w0, dev, nt, ns, args, rank, world, workspaces):
    """The same step through the public binding with HOST inputs and outputs: every step copies
    its inputs from pinned host memory and reads every result back, inside the timed region."""
    import torch
    amp, which = contrast_of(0, rank)
    wk = I.config_gaussian(amp, which, nt=nt, ns=ns)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_in = {"xa": pin(wk.xi_a), "xb": pin(wk.xi_b), "src": pin(wk.src_xy), "rec": pin(wk.rec_xy),
            "wav": pin(wk.wavelet)}
    nr = wk.nr
    h_data = torch.empty((ns, nr, nt), dtype=torch.float32).pin_memory()
    h_dtr = torch.empty_like(h_data).pin_memory()
    h_grads = torch.empty((5, 2, wk.nz, wk.nx), dtype=torch.float64).pin_memory()
    h_mis = torch.empty((), dtype=torch.float64).pin_memory()
    wm, wg, wb = workspaces
    h2d = sum(t.numel() * t.element_size() for t in h_in.values())
    d2h = sum(t.numel() * t.element_size() for t in (h_data, h_dtr, h_grads, h_mis))

    def step():
        d = {k: v.to(dev, non_blocking=True) for k, v in h_in.items()}
        zero = torch.zeros_like(d["xa"])
        data = fwi.fwi_model(g, w0.pz, d["xa"], d["xb"], d["src"], d["wav"], d["rec"], work=wm, check=False)
        mis, grads = fwi.fwi_gradient(g, w0.pz, zero, zero, d["src"], d["wav"], d["rec"], data, work=wg,
                                      check=False)
        dtr = fwi.fwi_born(g, w0.pz, zero, zero, d["xa"], d["xb"], d["src"], d["wav"], d["rec"], work=wb,
                           check=False)
        h_data.copy_(data, non_blocking=True)
        h_grads.copy_(grads, non_blocking=True)
        h_mis.copy_(mis, non_blocking=True)
        h_dtr.copy_(dtr, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    step()
    steps = max(1, min(args.steps, 5))   # up to 5 timed end-to-end steps (each ~2.7 s)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dt], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = t.item()
    upd = w0.Nx * w0.Nz * nt * ns * 4 * steps * world
    return {"value": round(upd / dt / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps}


if __name__ == "__main__":
    main()
