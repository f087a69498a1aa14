"""Error bowls (Sec. "Error-bowl Analysis"): the least-squares data misfit of a scatterer of
known shape as a function of its two contrasts, in each parameterization of Table 1.

For a known shape g(x) the model of parameterization pz is (xi_a, xi_b) = (a g, b g); every
grid point (a, b) is one forward solve, and the misfit J(a, b) = 1/2 |d(a, b) - d_obs|^2.  All
grid points run together as jobs of the batching engine (one batched launch per time step over
the whole grid), and each misfit is reduced by the library's fwi_misfit kernel.  The shape of a
bowl near its minimum -- how elongated it is and how it is oriented -- indicates how fast a
gradient method converges in that parameterization (circular: fast; elongated at 45 or 135
degrees: slow).

The scatterers of Table "tab:param_scat" whose shape is known: (i) point, vp only; (ii)
Gaussian, vp only; (iv) point, rho only; (v) Gaussian, rho only (the inversions of
``invert`` also take the unknown-shape ones, (iii), (vi) and (vii)).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import engine as E
from . import fwi as F
from . import inputs as I

CASES = {"i": ("point", "vp"), "ii": ("gaussian", "vp"), "iv": ("point", "rho"), "v": ("gaussian", "rho")}


def scatterer(case, amplitude=0.2, nt=1400):
    """The paper's acquisition (10 sources, 100 receivers on a 490 m circle, 5 Hz) around
    scatterer `case`; returns (workload with the true vp-rho contrasts, unit shape g)."""
    shape, which = CASES[case]
    w = I.config_paper(nt=nt, which=which, amplitude=amplitude)
    if shape == "point":
        g = I.point(w.nx, w.nz)
        z = np.zeros_like(g)
        w.xi_a, w.xi_b = (g * np.float32(amplitude), z) if which == "vp" else (z, g * np.float32(amplitude))
    else:
        g = I.gaussian(w.nx, w.nz, w.dx, I.centre_of(w.nx, w.nz, w.dx), 50.0)
    return w, g


# The scatterers of Table "tab:param_scat" whose shape is unknown to the inversion: (iii)
# Gaussian, vp only; (vi) Gaussian, rho only; (vii) Gaussian with no bulk-modulus contrast
# ((1 + xi_rho)(1 + xi_vp)^2 = 1, xi_vp the Gaussian).
UNKNOWN = {"iii": "vp", "vi": "rho", "vii": "nonK"}


def unknown_contrasts(g, kind, amplitude=0.2):
    """True (xi_vp, xi_rho) float32 fields of an unknown-shape scatterer of unit shape g."""
    a = (np.float32(amplitude) * g).astype(np.float32)
    z = np.zeros_like(a)
    if kind == "vp":
        return a, z
    if kind == "rho":
        return z, a
    return a, (1.0 / (1.0 + a.astype(np.float64)) ** 2 - 1.0).astype(np.float32)


def unknown_scatterer(case, amplitude=0.2, nt=1400):
    """The paper's acquisition around unknown-shape scatterer `case` (Gaussian, sigma 50 m):
    the workload with its true vp-rho contrasts."""
    w = I.config_paper(nt=nt, which="vp", amplitude=amplitude)
    g = I.gaussian(w.nx, w.nz, w.dx, I.centre_of(w.nx, w.nz, w.dx), 50.0)
    w.xi_a, w.xi_b = unknown_contrasts(g, UNKNOWN[case], amplitude)
    return w


def true_point(pz, dvp, drho):
    """Contrasts in parameterization pz of relative changes vp (1 + dvp), rho (1 + drho), from
    the exact relations of Table 2 (used only to centre the grid of a bowl)."""
    v, r = 1.0 + dvp, 1.0 + drho
    return {I.PZ_VP_RHO: (v - 1, r - 1), I.PZ_IP_RHO: (v * r - 1, r - 1), I.PZ_VP_IP: (v - 1, v * r - 1),
            I.PZ_K_RHO: (r * v * v - 1, r - 1), I.PZ_INVK_INVRHO: (1 / (r * v * v) - 1, 1 / r - 1)}[pz]


def grid_around(t, n=21, margin=1.0):
    """n evenly spaced contrasts that contain t itself and reach past both 0 (the starting
    model) and t by `margin` times max(|t|, 0.05)."""
    s = max(abs(t), 0.05)
    lo0, hi0 = min(0.0, t) - margin * s, max(0.0, t) + margin * s
    h = (hi0 - lo0) / (n - 1)
    m = int(round((t - lo0) / h))
    return t + h * (np.arange(n) - m)


def aperture_weights(src_xy, rec_xy, x0, lo_deg, hi_deg):
    """[ns][nr] float32 weights selecting the traces whose scattering angle at x0 -- the angle
    between the incident direction (source to x0) and the scattered one (x0 to receiver) --
    lies in [lo_deg, hi_deg] (Sec. "Hierarchical Inversion": short offsets 0-90 degrees, long
    offsets 135-180 degrees)."""
    s = np.asarray(src_xy, np.float64).reshape(-1, 2)
    r = np.asarray(rec_xy, np.float64).reshape(-1, 2)
    x0 = np.asarray(x0, np.float64)
    inc = x0 - s
    sca = r - x0
    inc /= np.linalg.norm(inc, axis=1, keepdims=True)
    sca /= np.linalg.norm(sca, axis=1, keepdims=True)
    ang = np.degrees(np.arccos(np.clip(inc @ sca.T, -1.0, 1.0)))
    return ((ang >= lo_deg) & (ang <= hi_deg)).astype(np.float32)


def error_bowl(w, g, pz, data, grid_a, grid_b, arena_bytes=None, work_budget=1 << 30, weights=None):
    """J[ia][ib] (float64 numpy) for contrasts (grid_a[ia] g, grid_b[ib] g) in parameterization
    pz against observed traces `data`; every grid point is a job of one engine.  weights:
    optional [ns][nr] trace weights (e.g. aperture_weights)."""
    dev = torch.device("cuda")
    grid = F.make_grid(**w.grid_kwargs())
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    src, rec, wav, gg = d(w.src_xy), d(w.rec_xy), d(w.wavelet), d(g)
    obs = F._dev(data).reshape(-1)
    wt = d(weights) if weights is not None else None
    if arena_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        arena_bytes = int(free * 0.5) // 256 * 256
    eng = E.Engine(arena_bytes)
    tick = {}
    with torch.cuda.stream(eng.stream):
        for ia, a in enumerate(grid_a):
            for ib, b in enumerate(grid_b):
                t = eng.submit_model(grid, pz, gg * float(a), gg * float(b), src, wav, rec, work_budget=work_budget)
                tick[t] = (ia, ib)
    J = torch.empty((len(grid_a), len(grid_b)), dtype=torch.float64, device=dev)
    launches = 0
    while tick:
        for r in eng.run(64):
            ia, ib = tick.pop(r.ticket)
            F.fwi_misfit(r.traces.reshape(-1), obs, misfit=J[ia, ib], stream=eng.stream, weights=wt, nt=w.nt)
        launches += F.launch_count()
    torch.cuda.synchronize()
    eng.close()
    return J.cpu().numpy(), launches


def bowl_shape(J, grid_a, grid_b, half=2):
    """Minimum, elongation and orientation of a bowl: a quadratic fitted by least squares to the
    (2 half + 1)^2 grid points around the smallest J.  Returns dict(argmin (a, b), J_min,
    condition = largest / smallest curvature, angle of the long axis in degrees from the a
    axis, in [0, 180))."""
    ia, ib = np.unravel_index(int(np.argmin(J)), J.shape)
    ia = int(np.clip(ia, half, J.shape[0] - 1 - half))
    ib = int(np.clip(ib, half, J.shape[1] - 1 - half))
    A, B, y = [], [], []
    for i in range(ia - half, ia + half + 1):
        for j in range(ib - half, ib + half + 1):
            A.append(grid_a[i] - grid_a[ia])
            B.append(grid_b[j] - grid_b[ib])
            y.append(J[i, j])
    A, B, y = map(np.asarray, (A, B, y))
    M = np.stack([np.ones_like(A), A, B, 0.5 * A * A, A * B, 0.5 * B * B], axis=1)
    c = np.linalg.lstsq(M, y, rcond=None)[0]
    H = np.array([[c[3], c[4]], [c[4], c[5]]])
    lam, vec = np.linalg.eigh(H)
    long_axis = vec[:, 0]                       # smallest curvature: the bowl's long axis
    angle = math.degrees(math.atan2(long_axis[1], long_axis[0])) % 180.0
    cond = float(lam[1] / lam[0]) if lam[0] > 0 else float("inf")
    i0, j0 = np.unravel_index(int(np.argmin(J)), J.shape)
    return dict(argmin=(float(grid_a[i0]), float(grid_b[j0])), J_min=float(J[i0, j0]), condition=cond,
                angle_deg=angle)


def born_error_bowl(acq, g, pz, data, grid_a, grid_b, scheme):
    """Schemes I/II: J[ia][ib] (float64 numpy) of the frequency-domain Born misfit for contrasts
    (grid_a[ia] g, grid_b[ib] g) of parameterization pz under the map of `scheme`, against
    data [nf][ns][nr] (fwi_fborn_misfit for every grid point)."""
    gg = torch.as_tensor(np.ascontiguousarray(g)).cuda()
    J = torch.empty((len(grid_a), len(grid_b)), dtype=torch.float64, device="cuda")
    for ia, a in enumerate(grid_a):
        for ib, b in enumerate(grid_b):
            acq.misfit(pz, gg * float(a), gg * float(b), data, scheme=scheme, out=J[ia, ib:ib + 1])
    return J.cpu().numpy()
