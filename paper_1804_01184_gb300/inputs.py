"""Seeded synthetic inputs shaped like the paper's experiments (arXiv:1804.01184).

This module is shared by the tests, the oracle checks and the benchmark.  It generates
inputs only -- contrast fields, acquisition geometry, the source wavelet, observed-data
stand-ins -- and holds none of the method's arithmetic (no parameter maps, stencils,
propagation or gradients).  Every array is returned in the precision the CUDA library
consumes (float32); the oracle receives the same values widened to float64, so both sides
see bit-identical inputs.

Workloads (the paper measures on no public dataset; these stand in for its synthetic
experiments, Sec. "Almost Well-posed Example" and the scatterer table):

  * ``config_point`` -- 201 x 201 nodes, dx 5 m, 4th order, dt 0.5 ms, 800 steps, 15 Hz
    Ricker, 8 sources / 64 receivers on a 400 m circle around the centre, 40-cell sponge
    outside the stated grid, point scatterer with +10 % K and +10 % rho (K-rho contrasts).
  * ``config_gaussian`` -- 601 x 601, dx 5 m, 8th order, 3000 steps, 64 sources / 256
    receivers on a 1200 m circle, Gaussian scatterer (sigma 20 m) in vp or rho only, contrast
    amplitude in [-0.5, 0.5] (vp-rho contrasts).
  * ``config_paper`` -- the paper's own acquisition: 10 sources, 100 receivers, 490 m
    circle, 5 Hz Ricker, vp = 2000 m/s, rho = 2000 kg/m^3, Gaussian sigma 50 m.
  * ``config_smooth`` -- 1201 x 1201, dx 2.5 m, dt 0.25 ms, 6000 steps, 16 sources / 256
    receivers on a 1200 m circle; smooth random background (seeded normal fields, Gaussian
    filter sigma 50 cells, min-max scaled to vp 1500-3500 m/s and rho 1000-2500 kg/m^3) plus
    4 Gaussian anomalies (sigma 25 m, +-20 % in vp and rho, centres in a 600 m disc).
  * ``batch_jobs`` -- uneven jobs for the batching and serving workloads: square grids with a
    side drawn uniformly from 128 to 1024 nodes (+ 40-cell sponge; dx 5 m, dt 0.5 ms, 8th
    order, 15 Hz), 500 to 4000 steps, 1 to 32 shots, 64 receivers, sources and receivers on a
    circle of radius 0.35 n dx, a point or Gaussian scatterer (sigma 10 to 40 m, each with
    probability 1/2) with contrasts drawn uniformly from [-0.5, 0.5] in vp and in rho.
  * ``poisson_arrivals`` -- seeded Poisson request times.
  * ``small_case`` -- seeded random heterogeneous models on small grids for parity tests.
  * ``freq_paper`` -- the frequency-domain Born workload of Schemes I/II: the paper's
    acquisition (10 sources, 100 receivers on a 490 m circle around x_0 = (0, 0), vp 2000 m/s,
    rho 2000 kg/m^3), a 121 x 121 model grid at dx 5 m centred on x_0 (inside the circle),
    the 5 Hz Ricker's spectrum at f_k = k 0.25 Hz, k = 1 .. 60, and a point or Gaussian
    (sigma 50 m) scatterer in vp or rho.
  * ``small_freq_case`` -- seeded random frequency-domain cases on small grids.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PZ_VP_RHO, PZ_IP_RHO, PZ_VP_IP, PZ_K_RHO, PZ_INVK_INVRHO = range(5)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    nz: int
    dx: float
    dt: float
    nt: int
    order: int
    sponge: int
    vp_o: float
    rho_o: float
    pz: int                 # parameterization of xi_a / xi_b
    xi_a: np.ndarray        # [nz][nx] float32 contrasts of the true model
    xi_b: np.ndarray
    src_xy: np.ndarray      # [ns][2] float32 metres, physical origin at node (0, 0)
    rec_xy: np.ndarray      # [nr][2] float32
    wavelet: np.ndarray     # [nt] float32, sample n at time (n + 1/2) dt
    sponge_v: float = 0.0   # 0 -> vp_o
    sponge_R: float = 1e-3

    @property
    def ns(self):
        return self.src_xy.shape[0]

    @property
    def nr(self):
        return self.rec_xy.shape[0]

    @property
    def Nx(self):
        return self.nx + 2 * self.sponge

    @property
    def Nz(self):
        return self.nz + 2 * self.sponge

    def cell_updates(self, shots=None):
        """Computational cells (sponge included) x steps x shots for one forward pass."""
        return self.Nx * self.Nz * self.nt * (self.ns if shots is None else shots)

    def background(self):
        z = np.zeros((self.nz, self.nx), np.float32)
        return z, z.copy()

    def grid_kwargs(self):
        return dict(nx=self.nx, nz=self.nz, dx=self.dx, dt=self.dt, nt=self.nt, order=self.order,
                    sponge=self.sponge, vp_o=self.vp_o, rho_o=self.rho_o,
                    sponge_v=self.sponge_v or self.vp_o, sponge_R=self.sponge_R)

    def subset(self, shots):
        """The same workload restricted to the listed shots."""
        w = dataclasses.replace(self)
        w.src_xy = np.ascontiguousarray(self.src_xy[list(shots)])
        return w


def ricker(nt, dt, f_peak, t0=None):
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0, t0 = 1/f,
    amplitude 1, sampled at t = (n + 1/2) dt (the time of the n-th source increment)."""
    t0 = 1.0 / f_peak if t0 is None else t0
    t = (np.arange(nt, dtype=np.float64) + 0.5) * dt - t0
    a = (math.pi * f_peak * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def circle(n, radius, centre, phase=0.0):
    """n points evenly on a circle, angles 2 pi (k + phase) / n, as float32 [n][2] (x, z)."""
    th = 2.0 * math.pi * (np.arange(n) + phase) / n
    xy = np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th)], axis=1)
    return xy.astype(np.float32)


def gaussian(nx, nz, dx, centre, sigma):
    """exp(-|x - x0|^2 / (2 sigma^2)) on the physical nodes, float32 [nz][nx]."""
    x = np.arange(nx) * dx - centre[0]
    z = np.arange(nz) * dx - centre[1]
    r2 = x[None, :] ** 2 + z[:, None] ** 2
    return np.exp(-r2 / (2.0 * sigma * sigma)).astype(np.float32)


def point(nx, nz):
    """One at the centre node, zero elsewhere, float32 [nz][nx]."""
    f = np.zeros((nz, nx), np.float32)
    f[nz // 2, nx // 2] = 1.0
    return f


def centre_of(nx, nz, dx):
    return ((nx - 1) * dx / 2.0, (nz - 1) * dx / 2.0)


def config_point(nt=800):
    nx = nz = 201
    dx = 5.0
    c = centre_of(nx, nz, dx)
    f = point(nx, nz) * np.float32(0.1)
    return Workload("point-201x201-o4", nx, nz, dx, 5e-4, nt, 4, 40, 2000.0, 2000.0, PZ_K_RHO,
                    f.copy(), f.copy(), circle(8, 400.0, c), circle(64, 400.0, c, 0.5),
                    ricker(nt, 5e-4, 15.0))


def config_gaussian(amplitude=0.3, which="vp", nt=3000, ns=64, nr=256, n=601):
    dx = 5.0
    c = centre_of(n, n, dx)
    g = gaussian(n, n, dx, c, 20.0) * np.float32(amplitude)
    z = np.zeros_like(g)
    xa, xb = (g, z) if which == "vp" else (z, g)
    radius = 1200.0 * (n - 1) / 600.0
    return Workload(f"gaussian-{n}x{n}-o8", n, n, dx, 5e-4, nt, 8, 40, 2000.0, 2000.0, PZ_VP_RHO,
                    xa, xb, circle(ns, radius, c), circle(nr, radius, c, 0.5),
                    ricker(nt, 5e-4, 15.0))


def config_paper(nt=1400, which="vp", amplitude=0.2):
    """The paper's acquisition: 10 sources, 100 receivers on a 490 m circle, 5 Hz, sigma 50 m."""
    dx = 10.0
    n = 121
    c = centre_of(n, n, dx)
    g = gaussian(n, n, dx, c, 50.0) * np.float32(amplitude)
    z = np.zeros_like(g)
    xa, xb = (g, z) if which == "vp" else (z, g)
    return Workload("paper-121x121-o8", n, n, dx, 1e-3, nt, 8, 40, 2000.0, 2000.0, PZ_VP_RHO,
                    xa, xb, circle(10, 490.0, c), circle(100, 490.0, c, 0.5),
                    ricker(nt, 1e-3, 5.0))


def config_smooth(nt=6000, ns=16, nr=256, n=1201, seed_vp=3, seed_rho=4, seed_anom=5):
    """Differentiation workload (vp-rho contrasts relative to vp_o = rho_o = 2000).  Returns the
    workload of the true model (background + anomalies) and the background contrasts."""
    from scipy.ndimage import gaussian_filter
    dx = 2.5
    c = centre_of(n, n, dx)

    def field(seed, lo, hi):
        f = gaussian_filter(np.random.default_rng(seed).standard_normal((n, n)), 50.0, mode="reflect")
        f = (f - f.min()) / (f.max() - f.min())
        return lo + (hi - lo) * f

    vp_bg, rho_bg = field(seed_vp, 1500.0, 3500.0), field(seed_rho, 1000.0, 2500.0)
    rng = np.random.default_rng(seed_anom)
    avp, arho = np.zeros((n, n)), np.zeros((n, n))
    for _ in range(4):
        r, th = 600.0 * np.sqrt(rng.random()), 2 * math.pi * rng.random()
        g = gaussian(n, n, dx, (c[0] + r * math.cos(th), c[1] + r * math.sin(th)), 25.0).astype(np.float64)
        avp += rng.uniform(-0.2, 0.2) * g
        arho += rng.uniform(-0.2, 0.2) * g
    vp, rho = vp_bg * (1 + avp), rho_bg * (1 + arho)
    w = Workload(f"smooth-{n}x{n}-o8", n, n, dx, 2.5e-4, nt, 8, 40, 2000.0, 2000.0, PZ_VP_RHO,
                 (vp / 2000.0 - 1).astype(np.float32), (rho / 2000.0 - 1).astype(np.float32),
                 circle(ns, 1200.0, c), circle(nr, 1200.0, c, 0.5), ricker(nt, 2.5e-4, 15.0),
                 sponge_v=4200.0)
    return w, ((vp_bg / 2000.0 - 1).astype(np.float32), (rho_bg / 2000.0 - 1).astype(np.float32))


def batch_job(seed, side=(128, 1024), steps=(500, 4000), shots=(1, 32)):
    """One uneven job of the batching/serving distribution (vp-rho contrasts of the true model)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(side[0], side[1] + 1))
    nt = int(rng.integers(steps[0], steps[1] + 1))
    ns = int(rng.integers(shots[0], shots[1] + 1))
    nr = 64
    dx, dt = 5.0, 5e-4
    c = centre_of(n, n, dx)
    if rng.random() < 0.5:
        shape = point(n, n)
    else:
        shape = gaussian(n, n, dx, c, float(rng.uniform(10.0, 40.0)))
    a, b = rng.uniform(-0.5, 0.5, size=2)
    radius = 0.35 * n * dx
    return Workload(f"job-{n}x{n}-o8-t{nt}-s{ns}", n, n, dx, dt, nt, 8, 40, 2000.0, 2000.0, PZ_VP_RHO,
                    (shape * np.float32(a)).astype(np.float32), (shape * np.float32(b)).astype(np.float32),
                    circle(ns, radius, c, float(rng.random())), circle(nr, radius, c, 0.5), ricker(nt, dt, 15.0))


def batch_jobs(count=256, seed=0, **kw):
    """`count` jobs of batch_job's distribution, job k seeded (seed, k)."""
    return [batch_job(np.random.SeedSequence([seed, k]), **kw) for k in range(count)]


def poisson_arrivals(count, rate, seed=0):
    """Arrival times (s) of a Poisson stream of `rate` requests per second."""
    return np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=count))


def small_case(seed=0, nx=45, nz=37, nt=120, order=8, sponge=6, ns=3, nr=7, pz=PZ_VP_RHO,
               amp=0.15, dx=5.0, dt=5e-4, f_peak=25.0):
    """Seeded heterogeneous model on a small grid: smooth random contrasts of size ~amp,
    sources and receivers at random positions inside the physical grid."""
    rng = np.random.default_rng(seed)

    def smooth():
        f = rng.standard_normal((nz, nx))
        for _ in range(3):   # a few passes of a 3-point box filter
            f = (np.roll(f, 1, 0) + f + np.roll(f, -1, 0)) / 3.0
            f = (np.roll(f, 1, 1) + f + np.roll(f, -1, 1)) / 3.0
        f /= max(1e-12, np.abs(f).max())
        return (amp * f).astype(np.float32)

    lo = np.array([2.0 * dx, 2.0 * dx])
    hi = np.array([(nx - 3) * dx, (nz - 3) * dx])
    src = (lo + (hi - lo) * rng.random((ns, 2))).astype(np.float32)
    rec = (lo + (hi - lo) * rng.random((nr, 2))).astype(np.float32)
    return Workload(f"small-{nx}x{nz}-o{order}-s{seed}", nx, nz, dx, dt, nt, order, sponge,
                    2000.0, 2000.0, pz, smooth(), smooth(), src, rec, ricker(nt, dt, f_peak))


def random_like(shape, seed, scale=1.0):
    """Seeded standard-normal float32 array (perturbations, residuals, test vectors)."""
    return (np.random.default_rng(seed).standard_normal(shape) * scale).astype(np.float32)


# ---------------------------------------------------------------- frequency-domain inputs

def ricker_spectrum(freqs, f_peak, t0=None):
    """Spectrum S(f) = integral w(t) e^{+i 2 pi f t} dt of the Ricker wavelet of peak f_peak
    delayed by t0 (default 1/f_peak), amplitude 1 (the e^{-i w t} convention):
    (2 / sqrt(pi)) (f^2 / f_peak^3) exp(-f^2 / f_peak^2) e^{i 2 pi f t0}; complex128."""
    t0 = 1.0 / f_peak if t0 is None else t0
    f = np.asarray(freqs, np.float64)
    amp = 2.0 / math.sqrt(math.pi) * f * f / f_peak ** 3 * np.exp(-(f / f_peak) ** 2)
    return amp * np.exp(2j * math.pi * f * t0)


@dataclasses.dataclass
class FreqWorkload:
    name: str
    nx: int
    nz: int
    dx: float
    x0: float               # coordinates of model node (0, 0)
    z0: float
    vp_o: float
    rho_o: float
    pz: int
    xi_a: np.ndarray        # [nz][nx] float32 contrasts of parameterization pz
    xi_b: np.ndarray
    src_xy: np.ndarray      # [ns][2] float32 metres
    rec_xy: np.ndarray      # [nr][2] float32
    freqs: np.ndarray       # [nf] float64 Hz
    spectrum: np.ndarray    # [nf] complex64 S(w_k)

    @property
    def ns(self):
        return self.src_xy.shape[0]

    @property
    def nr(self):
        return self.rec_xy.shape[0]

    @property
    def nf(self):
        return self.freqs.shape[0]

    def fgrid_kwargs(self):
        return dict(nx=self.nx, nz=self.nz, dx=self.dx, x0=self.x0, z0=self.z0, vp_o=self.vp_o,
                    rho_o=self.rho_o)

    def terms(self):
        """(frequency, source, receiver, node) terms of one pass over the data."""
        return self.nf * self.ns * self.nr * self.nx * self.nz

    def centre_index(self):
        return (self.nz // 2) * self.nx + self.nx // 2


def freq_paper(n=121, dx=5.0, which="vp", amplitude=0.2, shape="gaussian", nf=60, df=0.25,
               pz=PZ_VP_RHO, f_peak=5.0, ns=10, nr=100, radius=490.0):
    """The paper's almost well-posed example for the frequency-domain schemes; x_0 = (0, 0)
    is the centre node.  The contrasts are in vp-rho (parameterization A) unless pz says
    otherwise (the scatterer is then given in vp-rho and not converted: callers pass pz=0)."""
    h = (n - 1) / 2.0 * dx
    g = point(n, n) if shape == "point" else gaussian(n, n, dx, (h, h), 50.0)
    g = g * np.float32(amplitude)
    z = np.zeros_like(g)
    xa, xb = (g, z) if which == "vp" else (z, g)
    freqs = df * np.arange(1, nf + 1, dtype=np.float64)
    return FreqWorkload(f"freq-paper-{n}x{n}-{shape}-{which}", n, n, dx, -h, -h, 2000.0, 2000.0, pz, xa, xb,
                        circle(ns, radius, (0.0, 0.0)), circle(nr, radius, (0.0, 0.0), 0.5), freqs,
                        ricker_spectrum(freqs, f_peak).astype(np.complex64))


def small_freq_case(seed=0, nx=23, nz=19, dx=5.0, ns=3, nr=7, nf=5, amp=0.15, pz=PZ_VP_RHO,
                    radius=200.0, f_peak=8.0):
    """Seeded small frequency-domain case: smooth random contrasts of size ~amp on a grid
    centred at (0, 0), sources at random angles on a circle of `radius` outside the grid and
    receivers on one of 1.25 radius, random frequencies in (0.5 f_peak, 2.5 f_peak)."""
    rng = np.random.default_rng(seed)

    def smooth():
        f = rng.standard_normal((nz, nx))
        for _ in range(2):
            f = (np.roll(f, 1, 0) + f + np.roll(f, -1, 0)) / 3.0
            f = (np.roll(f, 1, 1) + f + np.roll(f, -1, 1)) / 3.0
        f /= max(1e-12, np.abs(f).max())
        return (amp * f).astype(np.float32)

    def ring(k, rad):
        th = 2.0 * math.pi * rng.random(k)
        return np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1).astype(np.float32)

    freqs = np.sort(f_peak * (0.5 + 2.0 * rng.random(nf)))
    return FreqWorkload(f"small-freq-{nx}x{nz}-s{seed}", nx, nz, dx, -(nx - 1) / 2.0 * dx, -(nz - 1) / 2.0 * dx,
                        2000.0, 2000.0, pz, smooth(), smooth(), ring(ns, radius), ring(nr, 1.25 * radius), freqs,
                        ricker_spectrum(freqs, f_peak).astype(np.complex64))
