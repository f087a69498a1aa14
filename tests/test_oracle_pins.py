"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test would fail on a plausible mistake in the oracle: a wrong stencil coefficient or
index (polynomial exactness, skew-adjointness, Green function), a wrong sign or dropped
term in the time step (energy, Green function), injection and sampling that are not
transposes (reciprocity), an adjoint that is not the transpose of Born (dot product), a
gradient or Born that is not the derivative of the forward model (Taylor, brute force),
parameter maps that disagree with Table 2, and a chain rule that is not the Jacobian of
the maps.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import hankel2

import oracle
from paper_1804_01184_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_of(w, **over):
    kw = w.grid_kwargs()
    kw.update(over)
    return oracle.make_grid(**kw)


# --------------------------------------------------------------------------- stencil

@pytest.mark.parametrize("order", [4, 8])
def test_coefficients_solve_taylor_conditions(order):
    """c_k of order 2M solve sum_k c_k (2k-1)^(2m-1) = [m == 1], m = 1..M (exact fractions)."""
    M = order // 2
    A = [[Fraction(2 * k - 1) ** (2 * m - 1) for k in range(1, M + 1)] for m in range(1, M + 1)]
    b = [Fraction(1 if m == 0 else 0) for m in range(M)]
    # Gauss-Jordan in exact arithmetic
    for col in range(M):
        piv = A[col][col]
        A[col] = [a / piv for a in A[col]]
        b[col] /= piv
        for r in range(M):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * p for a, p in zip(A[r], A[col])]
                b[r] -= f * b[col]
    np.testing.assert_allclose(oracle.coefficients(order), [float(x) for x in b], rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("minus", [0, 1])
def test_stencil_exact_on_polynomials(order, minus):
    """D+ (node -> half node) and D- (half node -> node) differentiate polynomials of degree
    < order exactly away from the ends; the evaluation point is shifted by half a cell."""
    n, dx, M = 40, 0.7, order // 2
    for deg in range(order):
        pos = np.arange(n) * dx + (0.5 * dx if minus else 0.0)   # where the input lives
        f = (pos / 10.0) ** deg
        out = oracle.apply_d(f, order, minus, dx)
        ev = np.arange(n) * dx + (0.0 if minus else 0.5 * dx)    # where the output lives
        exact = deg * (ev / 10.0) ** max(deg - 1, 0) / 10.0 if deg > 0 else 0 * ev
        sl = slice(M, n - M)
        np.testing.assert_allclose(out[sl], exact[sl], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("order", [4, 8])
def test_dminus_is_minus_transpose_of_dplus(order):
    n = 23
    Dp = np.stack([oracle.apply_d(e, order, 0) for e in np.eye(n)], axis=1)
    Dm = np.stack([oracle.apply_d(e, order, 1) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(Dm, -Dp.T, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ parameterizations

def table2(xK, xr):
    """Table 2 of the paper: contrasts of pairs (A)-(D) from (xi_{1/K}, xi_{1/rho})."""
    vp = math.sqrt((xr + 1) / (xK + 1)) - 1
    Ip = math.sqrt(1 / ((xr + 1) * (xK + 1))) - 1
    rho = -xr / (xr + 1)
    K = -xK / (xK + 1)
    return {0: (vp, rho), 1: (Ip, rho), 2: (vp, Ip), 3: (K, rho)}


def test_forward_maps_agree_with_table2():
    rng = np.random.default_rng(7)
    for _ in range(50):
        xK, xr = rng.uniform(-0.6, 0.8, 2)
        K_e, r_e = oracle.forward_map(4, xK, xr)
        for pz, (a, b) in table2(xK, xr).items():
            K, r = oracle.forward_map(pz, a, b)
            assert abs(K - K_e) <= 1e-12 * K_e and abs(r - r_e) <= 1e-12 * r_e


def test_forward_map_rejects_nonpositive():
    with pytest.raises(ValueError):
        oracle.forward_map(0, -1.0, 0.0)
    with pytest.raises(ValueError):
        oracle.forward_map(4, 0.0, -1.5)


def test_chain_rule_is_jacobian_of_maps():
    """Chain-rule output vs central differences of the forward maps, at random models."""
    rng = np.random.default_rng(8)
    vp_o, rho_o = 2000.0, 2000.0
    n = 20
    K = vp_o ** 2 * rho_o * rng.uniform(0.5, 1.8, n)
    rho = rho_o * rng.uniform(0.6, 1.5, n)
    gK, grho = rng.standard_normal(n), rng.standard_normal(n)
    G = oracle.chain_rule(vp_o, rho_o, K, rho, gK * 1e-9, grho)
    # contrasts of the same model in each pair, by Table 1's definitions
    vp, Ip = np.sqrt(K / rho), np.sqrt(K * rho)
    ab = {0: (vp / vp_o - 1, rho / rho_o - 1), 1: (Ip / (rho_o * vp_o) - 1, rho / rho_o - 1),
          2: (vp / vp_o - 1, Ip / (rho_o * vp_o) - 1), 3: (K / (rho_o * vp_o ** 2) - 1, rho / rho_o - 1),
          4: (rho_o * vp_o ** 2 / K - 1, rho_o / rho - 1)}
    h = 1e-6
    for pz in range(5):
        for c in range(n):
            a, b = ab[pz][0][c], ab[pz][1][c]
            for which in range(2):
                da, db = (h, 0) if which == 0 else (0, h)
                Kp, rp = oracle.forward_map(pz, a + da, b + db, vp_o, rho_o)
                Km, rm = oracle.forward_map(pz, a - da, b - db, vp_o, rho_o)
                fd = (Kp - Km) / (2 * h) * gK[c] * 1e-9 + (rp - rm) / (2 * h) * grho[c]
                assert abs(G[pz, which, c] - fd) <= 1e-6 * (abs(fd) + 1e-3 * abs(G[pz, which, c]) + 1e-3)


def test_model_build_buoyancy_and_padding():
    w = I.small_case(seed=3, nx=9, nz=7, sponge=3)
    g = grid_of(w)
    K, rho, bx, bz = oracle.model_build(g, w.pz, w.xi_a, w.xi_b)
    S = w.sponge
    # padding copies the nearest physical cell
    np.testing.assert_array_equal(rho[:S, S:-S], np.repeat(rho[S:S + 1, S:-S], S, 0))
    np.testing.assert_array_equal(K[S:-S, -S:], np.repeat(K[S:-S, -S - 1:-S], S, 1))
    # buoyancy: 2 / (rho_i + rho_{i+1}), the last node reuses its own rho
    np.testing.assert_allclose(bx[:, :-1], 2 / (rho[:, :-1] + rho[:, 1:]), rtol=1e-15)
    np.testing.assert_allclose(bx[:, -1], 1 / rho[:, -1], rtol=1e-15)
    np.testing.assert_allclose(bz[:-1], 2 / (rho[:-1] + rho[1:]), rtol=1e-15)
    # vp-rho map (Table 1): K = rho vp^2
    vp = 2000.0 * (1 + w.xi_a.astype(np.float64))
    np.testing.assert_allclose(K[S:-S, S:-S], 2000.0 * (1 + w.xi_b.astype(np.float64)) * vp ** 2, rtol=1e-14)


def test_sponge_profile():
    d = oracle.sponge_profile(10, 5, 5.0, 5e-4, 2000.0, 1e-3, 0)
    assert np.all(d[5:15] == 1.0)
    assert np.all(np.diff(d[:6]) > 0) and np.all(np.diff(d[14:]) < 0)
    smax = 3 * 2000.0 * math.log(1e3) / (2 * 5 * 5.0)
    assert abs(d[0] - math.exp(-smax * 5e-4)) < 1e-15
    np.testing.assert_allclose(d, d[::-1], rtol=0, atol=0)
    dh = oracle.sponge_profile(10, 5, 5.0, 5e-4, 2000.0, 1e-3, 1)
    np.testing.assert_allclose(dh[:-1], dh[:-1][::-1], rtol=1e-15)
    assert np.all(oracle.sponge_profile(10, 0, 5.0, 5e-4, 2000.0, 1e-3, 0) == 1.0)


def test_bilinear_weights():
    g = oracle.make_grid(11, 9, 5.0, 5e-4, 10, sponge=2)
    idx, w = oracle.weights(g, 12.5, 6.0)
    Nx = 11 + 4
    assert idx[0] == (1 + 2) * Nx + (2 + 2)
    np.testing.assert_allclose(w, [0.5 * 0.8, 0.5 * 0.8, 0.5 * 0.2, 0.5 * 0.2], rtol=1e-14)
    assert abs(w.sum() - 1) < 1e-15
    idx, w = oracle.weights(g, 50.0, 40.0)          # last physical node: all weight there
    assert w[idx == (8 + 2) * Nx + (10 + 2)].sum() == 1.0
    with pytest.raises(ValueError):
        oracle.weights(g, 50.1, 0.0)


# ------------------------------------------------------------------- physics pins

def ricker_continuous(t, f, t0):
    a = (math.pi * f * (t - t0)) ** 2
    return (1 - 2 * a) * np.exp(-a)


def green_trace(r, c, rho, f, t0, t_out):
    """Pressure of p_tt - c^2 lap p = K d/dt[w(t)] delta(x) (volume injection rate w) at
    distance r: P(w) = rho w W(w) H0^(2)(w r / c) / 4 with numpy's FFT sign (the conjugate
    of the e^{-iwt} form i/4 H0^(1) of the 2-D Green function of the paper's reference
    operator)."""
    dtf, N = 1e-5, 1 << 18
    t = np.arange(N) * dtf
    W = np.fft.rfft(ricker_continuous(t, f, t0)) * dtf
    om = 2 * np.pi * np.fft.rfftfreq(N, dtf)
    P = np.zeros_like(W)
    P[1:] = rho * om[1:] * W[1:] * hankel2(0, om[1:] * r / c) / 4
    return np.interp(t_out, t, np.fft.irfft(P, N) / dtf)


def test_homogeneous_green_function_convergence():
    """Homogeneous medium: traces vs the analytic 2-D Green function convolved with the
    Ricker, before any boundary arrival; error falls at 2nd order under joint (dx, dt)
    refinement and is below 1 % at dx = 2.5 m (8th order)."""
    f, t0, r, L = 15.0, 1.5 / 15.0, 300.0, 1000.0
    errs = []
    for dx, dt in ((10.0, 1e-3), (5.0, 5e-4), (2.5, 2.5e-4)):
        n, nt = int(L / dx) + 1, int(round(0.4 / dt))
        g = oracle.make_grid(n, n, dx, dt, nt, order=8, sponge=int(200 / dx))
        z = np.zeros((n, n))
        src = np.array([[L / 2, L / 2]])
        rec = np.array([[L / 2 + r, L / 2]])
        tr = oracle.model(g, 3, z, z, src, I.ricker(nt, dt, f, t0), rec)[0, 0]
        pa = green_trace(r, 2000.0, 2000.0, f, t0, (np.arange(nt) + 1) * dt)
        errs.append(np.linalg.norm(tr - pa) / np.linalg.norm(pa))
    assert errs[2] < 1e-2
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_reciprocity_heterogeneous_with_sponge():
    w = I.small_case(seed=2, nx=45, nz=37, nt=200, sponge=8, ns=2, nr=2, pz=I.PZ_IP_RHO)
    g = grid_of(w)
    A, B = w.src_xy[:1], w.src_xy[1:2]
    tAB = oracle.model(g, w.pz, w.xi_a, w.xi_b, A, w.wavelet, B)
    tBA = oracle.model(g, w.pz, w.xi_a, w.xi_b, B, w.wavelet, A)
    assert np.abs(tAB - tBA).max() <= 1e-12 * np.abs(tAB).max()


def test_discrete_energy_conserved_without_sponge():
    w = I.small_case(seed=1, nx=41, nz=41, nt=2500, sponge=0, ns=1, nr=1)
    g = grid_of(w)
    E = oracle.energy(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet)
    assert np.abs(w.wavelet[300:]).max() < 1e-20          # source has ended
    assert np.abs(E[300:] - E[300]).max() <= 1e-12 * E[300]
    w.sponge = 6
    E = oracle.energy(grid_of(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet)
    assert np.all(np.diff(E[300:]) <= 1e-12 * E[300]) and E[-1] < 1e-3 * E[300]


def test_d4_symmetry_point_scatterer():
    """Square grid, centred scatterer, sources every 45 deg and receivers offset by half a
    spacing: a 90-degree rotation maps shot s to s+2 and receiver r to r+16.  The staggered
    grid's outermost half node (N - 1/2) has no mirror at -1/2, so the record ends before any
    wave can reach the padded edge and come back (edge 150 m from the ring, 100 ms record)."""
    n, dx = 81, 5.0
    c = (n - 1) * dx / 2
    th_s = 2 * np.pi * np.arange(8) / 8
    th_r = 2 * np.pi * (np.arange(64) + 0.5) / 64
    R = 80.0
    # exact rotation images: build one quadrant and rotate offsets by (x, z) -> (-z, x)
    def ring(th, n_per_q):
        q = np.stack([R * np.cos(th[:n_per_q]), R * np.sin(th[:n_per_q])], 1)
        out = [q]
        for _ in range(3):
            q = np.stack([-q[:, 1], q[:, 0]], 1)
            out.append(q)
        return np.concatenate(out) + c
    src, rec = ring(th_s, 2), ring(th_r, 16)
    xi = np.zeros((n, n))
    xi[n // 2, n // 2] = 0.2
    g = oracle.make_grid(n, n, dx, 5e-4, 200, order=4, sponge=6)
    tr = oracle.model(g, 3, xi, xi, src, I.ricker(200, 5e-4, 25.0), rec)
    rot = tr[(np.arange(8) + 2) % 8][:, (np.arange(64) + 16) % 64]
    assert np.abs(tr - rot).max() <= 1e-10 * np.abs(tr).max()


# -------------------------------------------------------------- adjoint / gradient

@pytest.mark.parametrize("pz", range(5))
def test_dot_product_born_adjoint(pz):
    w = I.small_case(seed=3, pz=pz, nt=100)
    g = grid_of(w)
    da, db = I.random_like(w.xi_a.shape, 10), I.random_like(w.xi_a.shape, 11)
    y = I.random_like((w.ns, w.nr, w.nt), 12)
    Fx = oracle.born(g, pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
    G = oracle.adjoint(g, pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, y)
    lhs, rhs = np.sum(Fx * y), np.sum(G[pz, 0] * da) + np.sum(G[pz, 1] * db)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("pz", range(5))
def test_taylor_gradient(pz):
    w = I.small_case(seed=4, pz=pz, nt=100)
    g = grid_of(w)
    d_obs = oracle.model(g, pz, w.xi_a * 1.3, w.xi_b * 0.7, w.src_xy, w.wavelet, w.rec_xy)
    a0, b0 = w.xi_a * 0.5, w.xi_b * 0.5
    J0, G = oracle.gradient(g, pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, d_obs)
    da, db = I.random_like(a0.shape, 20, 0.05), I.random_like(a0.shape, 21, 0.05)
    lin = np.sum(G[pz, 0] * da) + np.sum(G[pz, 1] * db)
    hs = [0.1 / 2 ** k for k in range(6)]
    r = []
    for h in hs:
        Jh, _ = oracle.gradient(g, pz, a0 + h * da, b0 + h * db, w.src_xy, w.wavelet, w.rec_xy, d_obs)
        r.append(abs(Jh - J0 - h * lin))
    slopes = np.log2(np.array(r[:-1]) / np.array(r[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


@pytest.mark.parametrize("pz", [0, 4])
def test_taylor_born(pz):
    w = I.small_case(seed=5, pz=pz, nt=100)
    g = grid_of(w)
    da, db = I.random_like(w.xi_a.shape, 30, 0.05), I.random_like(w.xi_a.shape, 31, 0.05)
    d0 = oracle.model(g, pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    F = oracle.born(g, pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
    r = []
    for h in [0.1 / 2 ** k for k in range(6)]:
        dh = oracle.model(g, pz, w.xi_a + h * da, w.xi_b + h * db, w.src_xy, w.wavelet, w.rec_xy)
        r.append(np.linalg.norm(dh - d0 - h * F))
    slopes = np.log2(np.array(r[:-1]) / np.array(r[1:]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), slopes


def test_brute_force_gradient_tiny_grid():
    """Central differences of J w.r.t. every contrast component (21 x 21 grid, 60 steps)."""
    w = I.small_case(seed=6, nx=21, nz=21, nt=60, sponge=4, ns=2, nr=5, pz=I.PZ_VP_RHO, f_peak=40.0)
    g = grid_of(w)
    d_obs = oracle.model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    rng = np.random.default_rng(0)
    for pz in range(5):
        a0 = (rng.standard_normal(w.xi_a.shape) * 0.05).astype(np.float64)
        b0 = (rng.standard_normal(w.xi_a.shape) * 0.05).astype(np.float64)
        J0, G = oracle.gradient(g, pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, d_obs)
        cells = [(j, i) for j in range(21) for i in range(21)] if pz in (0, 3) else \
            [tuple(x) for x in rng.integers(0, 21, (25, 2))]
        h = 1e-4
        for which in range(2):
            for (j, i) in cells:
                a, b = a0.copy(), b0.copy()
                (a if which == 0 else b)[j, i] += h
                Jp = oracle_misfit(g, pz, a, b, w, d_obs)
                (a if which == 0 else b)[j, i] -= 2 * h
                Jm = oracle_misfit(g, pz, a, b, w, d_obs)
                fd = (Jp - Jm) / (2 * h)
                scale = np.abs(G[pz, which]).max()
                assert abs(G[pz, which, j, i] - fd) <= 1e-7 * scale + 1e-6 * abs(fd), (pz, which, j, i)


def oracle_misfit(g, pz, a, b, w, d_obs):
    tr = oracle.model(g, pz, a, b, w.src_xy, w.wavelet, w.rec_xy)
    return 0.5 * np.sum((tr - d_obs) ** 2)


def test_gradient_misfit_and_zero_residual():
    w = I.small_case(seed=9, pz=I.PZ_K_RHO, nt=80)
    g = grid_of(w)
    d = oracle.model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    J, G = oracle.gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, d)
    assert J == 0.0 and np.all(G == 0.0)
    d2 = d + I.random_like(d.shape, 3, 1.0)
    J2, _ = oracle.gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, d2)
    assert abs(J2 - 0.5 * np.sum((d - d2) ** 2)) <= 1e-12 * J2


def test_paper_acquisition_fixture():
    """The paper-shape workload reproduces the paper's stated setup (golden fixture)."""
    with open(os.path.join(GOLDEN, "paper_setup.json")) as fh:
        gold = json.load(fh)
    w = I.config_paper()
    assert w.ns == gold["n_sources"] and w.nr == gold["n_receivers"]
    c = np.array(I.centre_of(w.nx, w.nz, w.dx))
    for xy in (w.src_xy, w.rec_xy):
        np.testing.assert_allclose(np.linalg.norm(xy - c, axis=1), gold["circle_radius_m"], rtol=1e-6)
    assert w.vp_o == gold["vp_background_m_per_s"] and w.rho_o == gold["rho_background_kg_per_m3"]
    assert gold["vp_background_m_per_s"] / gold["ricker_peak_hz"] == gold["dominant_wavelength_m"]
    # the Ricker peaks at t0 = 1/f with amplitude 1
    k = int(np.argmax(w.wavelet))
    assert abs((k + 0.5) * w.dt - 1.0 / gold["ricker_peak_hz"]) <= w.dt and w.wavelet.max() <= 1.0
