"""Pins of the frequency-domain Born oracle (Schemes I/II) against what the paper and the
mathematics fix: the Green function's equation, normalization and outgoing direction; the
printed re-parameterization tables; the finite-difference time-domain modelling of Scheme III
(the Born scattered field of a weak scatterer); Taylor tests of the gradient; the Hessian as
the difference of gradients; and the paper's statement that only the K-rho and 1/K-1/rho
reduced Hessians have no cross-parameter term for a full circular acquisition."""
import math

import numpy as np
import pytest
from scipy.special import hankel1

import oracle
from oracle import fborn as FB
from paper_1804_01184_gb300 import inputs as I


def fgrid(w):
    return FB.FGrid(**w.fgrid_kwargs())


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# ---------------------------------------------------------------- Green function

def test_green_solves_helmholtz_away_from_source():
    """(lap + k^2) G_o = 0 off the source: a 5-point Laplacian with h = 0.25 m leaves a
    residual of O((k h)^2) relative to k^2 |G|."""
    fg = FB.FGrid(3, 3, 1.0, 0.0, 0.0, vp_o=1800.0, rho_o=2300.0)
    for f, x, z in ((7.0, 130.0, 40.0), (15.0, -60.0, 210.0), (3.0, 35.0, -20.0)):
        k = 2 * math.pi * f / fg.vp_o
        h = 0.25
        G = lambda dx, dz: FB.green(fg, f, math.hypot(x + dx, z + dz))[0]
        lap = (G(h, 0) + G(-h, 0) + G(0, h) + G(0, -h) - 4 * G(0, 0)) / h ** 2
        assert abs(lap + k * k * G(0, 0)) < 1e-4 * k * k * abs(G(0, 0))


def test_green_radial_derivative():
    fg = FB.FGrid(3, 3, 1.0, 0.0, 0.0)
    for f, r in ((5.0, 80.0), (12.0, 333.0)):
        h = 1e-3
        num = (FB.green(fg, f, r + h)[0] - FB.green(fg, f, r - h)[0]) / (2 * h)
        assert abs(num - FB.green(fg, f, r)[1]) < 1e-7 * abs(num)


def test_green_normalization_and_sign():
    """Flux of (1/rho_o) grad G_o through a small circle: -1 (the reading L_o G_o = -delta that
    makes the printed Lippmann-Schwinger equation exact), for any frequency and medium."""
    for vp, rho, f in ((2000.0, 2000.0, 5.0), (1500.0, 1000.0, 20.0)):
        fg = FB.FGrid(3, 3, 1.0, 0.0, 0.0, vp_o=vp, rho_o=rho)
        eps = 1e-5
        flux = 2 * math.pi * eps / rho * FB.green(fg, f, eps)[1]
        assert abs(flux - (-1.0)) < 1e-6


def test_green_is_outgoing():
    """Far field: G(r + d) / G(r) -> sqrt(r / (r + d)) e^{+i k d} (outgoing for e^{-i w t})."""
    fg = FB.FGrid(3, 3, 1.0, 0.0, 0.0)
    f, r, d = 20.0, 5000.0, 17.0
    k = 2 * math.pi * f / fg.vp_o
    ratio = FB.green(fg, f, r + d)[0] / FB.green(fg, f, r)[0]
    assert abs(ratio - math.sqrt(r / (r + d)) * np.exp(1j * k * d)) < 1e-4


def test_modelling_vectors_reciprocal():
    """W(x; x_r, x_s) = W(x; x_s, x_r): swapping sources and receivers transposes W."""
    w = I.small_freq_case(seed=2)
    fg = fgrid(w)
    W = FB.modelling_vectors(fg, w.freqs[1], w.src_xy, w.rec_xy)
    Wt = FB.modelling_vectors(fg, w.freqs[1], w.rec_xy, w.src_xy)
    np.testing.assert_allclose(W, np.transpose(Wt, (1, 0, 2, 3)), rtol=1e-13, atol=0)


def test_ricker_spectrum_matches_fft_of_the_wavelet():
    f_peak, t0, dt, n = 5.0, 0.5, 1e-3, 1 << 14
    t = np.arange(n) * dt
    a = (math.pi * f_peak * (t - t0)) ** 2
    w = (1 - 2 * a) * np.exp(-a)
    F = np.conj(np.fft.rfft(w)) * dt            # e^{+i 2 pi f t} transform
    fr = np.fft.rfftfreq(n, dt)
    sel = (fr > 0.5) & (fr < 15)
    np.testing.assert_allclose(F[sel], I.ricker_spectrum(fr[sel], f_peak, t0), atol=1e-9)


# ---------------------------------------------------------------- re-parameterizations

TABLE2 = {   # Table 2 as printed: (xi_a, xi_b) of pz from (x1, x2) = (xi_{1/K}, xi_{1/rho})
    0: lambda x1, x2: (np.sqrt((x2 + 1) / (x1 + 1)) - 1, -x2 / (x2 + 1)),
    1: lambda x1, x2: (np.sqrt(1 / ((x2 + 1) * (x1 + 1))) - 1, -x2 / (x2 + 1)),
    2: lambda x1, x2: (np.sqrt((x2 + 1) / (x1 + 1)) - 1, np.sqrt(1 / ((x2 + 1) * (x1 + 1))) - 1),
    3: lambda x1, x2: (-x1 / (x1 + 1), -x2 / (x2 + 1)),
}


@pytest.mark.parametrize("pz", [0, 1, 2, 3])
def test_exact_map_inverts_table2(pz):
    rng = np.random.default_rng(pz)
    a, b = rng.uniform(-0.5, 0.5, 50), rng.uniform(-0.5, 0.5, 50)
    x1, x2 = FB.to_inverse_contrasts(pz, a, b, FB.NONLINEAR)
    ra, rb = TABLE2[pz](x1, x2)
    np.testing.assert_allclose(ra, a, atol=1e-13)
    np.testing.assert_allclose(rb, b, atol=1e-13)


def test_exact_map_of_inverse_parameterization_is_identity():
    a, b = np.array([0.3, -0.2]), np.array([-0.1, 0.4])
    x1, x2 = FB.to_inverse_contrasts(4, a, b, FB.NONLINEAR)
    np.testing.assert_array_equal(x1, a)
    np.testing.assert_array_equal(x2, b)


@pytest.mark.parametrize("pz", range(5))
def test_linear_map_is_jacobian_of_exact_map_at_zero(pz):
    h = 1e-7
    L = FB.linear_jacobian(pz)
    for k, (da, db) in enumerate(((h, 0.0), (0.0, h))):
        p = np.array(FB.to_inverse_contrasts(pz, da, db, FB.NONLINEAR))
        m = np.array(FB.to_inverse_contrasts(pz, -da, -db, FB.NONLINEAR))
        np.testing.assert_allclose((p - m) / (2 * h), L[:, k], atol=1e-7)


def test_linear_map_inverts_table3():
    """Table 3 as printed for the vp, rho, K rows; for the Ip rows the printed
    xi_{1/rho} - xi_{1/K}/2 fails and the linearization of Table 2, -(xi_{1/K} + xi_{1/rho})/2,
    holds (reading F5)."""
    a, b = 0.013, -0.021
    vp_row = lambda x1, x2: 0.5 * (x2 - x1)
    ip_printed = lambda x1, x2: x2 - 0.5 * x1
    ip_linear = lambda x1, x2: -0.5 * (x1 + x2)
    x1, x2 = FB.to_inverse_contrasts(0, a, b, FB.LINEAR)
    assert abs(vp_row(x1, x2) - a) < 1e-15 and abs(-x2 - b) < 1e-15
    x1, x2 = FB.to_inverse_contrasts(3, a, b, FB.LINEAR)
    assert abs(-x1 - a) < 1e-15 and abs(-x2 - b) < 1e-15
    x1, x2 = FB.to_inverse_contrasts(2, a, b, FB.LINEAR)
    assert abs(vp_row(x1, x2) - a) < 1e-15 and abs(ip_linear(x1, x2) - b) < 1e-15
    assert abs(ip_printed(x1, x2) - b) > 1e-3
    x1, x2 = FB.to_inverse_contrasts(1, a, b, FB.LINEAR)
    assert abs(ip_linear(x1, x2) - a) < 1e-15 and abs(-x2 - b) < 1e-15
    assert abs(ip_printed(x1, x2) - a) > 1e-3


@pytest.mark.parametrize("pz", range(5))
def test_exact_map_jacobian_matches_finite_differences(pz):
    rng = np.random.default_rng(10 + pz)
    a, b = rng.uniform(-0.4, 0.4, 7), rng.uniform(-0.4, 0.4, 7)
    J = FB.jacobian(pz, a, b, FB.NONLINEAR)
    h = 1e-6
    for k in range(2):
        da, db = (h, 0.0) if k == 0 else (0.0, h)
        p = np.array(FB.to_inverse_contrasts(pz, a + da, b + db, FB.NONLINEAR))
        m = np.array(FB.to_inverse_contrasts(pz, a - da, b - db, FB.NONLINEAR))
        np.testing.assert_allclose((p - m) / (2 * h), J[:, k], rtol=1e-6, atol=1e-8)


# ---------------------------------------------------------------- Born vs Scheme III

def test_born_matches_time_domain_scattered_field():
    """A weak Gaussian scatterer (xi_{1/K} = +1 %, xi_{1/rho} = +0.5 %, sigma 20 m): the
    Born scattered field of the frequency-domain oracle, taken to the time domain with the
    injected Ricker, equals the scattered field of the finite-difference oracle (Scheme III:
    run with the scatterer minus run without) at receivers in forward, side, oblique and
    back scattering, to the FD and Born errors (measured: 0.5 - 1.3 %, bound 3 %).  A flipped
    or missing density term, a wrong w^2/K_o or 1/rho_o factor or a lost dx^2 fails it."""
    dx, dt, nt, f_peak, sp = 5.0, 5e-4, 1200, 10.0, 40
    n = 161
    c = (400.0, 400.0)
    g = oracle.make_grid(n, n, dx, dt, nt, order=8, sponge=sp)
    gau = I.gaussian(n, n, dx, c, 20.0).astype(np.float64)
    x1, x2 = 0.01 * gau, 0.005 * gau
    z = np.zeros_like(x1)
    src = np.array([[400.0, 100.0]])
    rec = np.array([[400.0, 700.0], [700.0, 400.0], [612.0, 612.0], [440.0, 100.0]])
    wav = I.ricker(nt, dt, f_peak).astype(np.float64)
    fd = oracle.model(g, 4, x1, x2, src, wav, rec)[0] - oracle.model(g, 4, z, z, src, wav, rec)[0]
    # Born: the model grid is the FD nodes within 100 m of the scatterer
    m = 41
    fg = FB.FGrid(m, m, dx, c[0] - 100.0, c[1] - 100.0)
    i0 = int(round((c[0] - 100.0) / dx))
    xi = np.stack([x1[i0:i0 + m, i0:i0 + m].ravel(), x2[i0:i0 + m, i0:i0 + m].ravel()], axis=-1)
    N = 4096
    fr = np.fft.rfftfreq(N, dt)
    t0 = 1.0 / f_peak
    Pall = np.zeros((len(rec), fr.size), np.complex128)
    for k in range(1, np.searchsorted(fr, 50.0)):
        W = FB.modelling_vectors(fg, fr[k], src, rec)[0]           # [nr][N][2]
        Ws = np.einsum("rnc,nc->r", W, xi) * dx * dx
        # FD source: volume-injection rate w(t) -> pressure S = -i w W(w) (e^{-iwt}); the
        # real trace's numpy spectrum is the conjugate
        S = -1j * 2 * math.pi * fr[k] * I.ricker_spectrum(fr[k], f_peak, t0)
        Pall[:, k] = np.conj(S * Ws)
    born = np.fft.irfft(Pall, N, axis=1) / dt                        # sample m at time m dt
    born = born[:, 1:nt + 1]                                           # FD sample n at (n+1) dt
    for r in range(len(rec)):
        e = rel(fd[r], born[r])
        assert e < 0.03, (r, e)
    # the density term matters: without it the forward and back receivers are far off
    xi_k = xi.copy()
    xi_k[:, 1] = 0.0
    for k in range(1, np.searchsorted(fr, 50.0)):
        W = FB.modelling_vectors(fg, fr[k], src, rec)[0]
        S = -1j * 2 * math.pi * fr[k] * I.ricker_spectrum(fr[k], f_peak, t0)
        Pall[:, k] = np.conj(S * np.einsum("rnc,nc->r", W, xi_k) * dx * dx)
    bk = (np.fft.irfft(Pall, N, axis=1) / dt)[:, 1:nt + 1]
    assert rel(fd[0], bk[0]) > 0.3 and rel(fd[3], bk[3]) > 0.3


# ---------------------------------------------------------------- gradient and Hessian

@pytest.mark.parametrize("scheme", [FB.LINEAR, FB.NONLINEAR])
@pytest.mark.parametrize("pz", range(5))
def test_gradient_taylor(pz, scheme):
    """J(m + e d) - J(m) - e <g, d> falls as e^2 (second order) for both schemes."""
    w = I.small_freq_case(seed=3 + pz, pz=pz, nx=9, nz=8, ns=2, nr=4, nf=3)
    fg = fgrid(w)
    q = FB.model(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, w.xi_a * 1.3, w.xi_b * 0.7, FB.NONLINEAR)
    a0, b0 = w.xi_a.astype(np.float64), w.xi_b.astype(np.float64)
    J0, ga, gb = FB.gradient(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a0, b0, q, scheme)
    rng = np.random.default_rng(pz)
    da, db = rng.standard_normal(a0.shape), rng.standard_normal(b0.shape)
    slope = float(np.sum(ga * da) + np.sum(gb * db))
    errs = []
    for e in (1e-2, 5e-3, 2.5e-3):
        Je = FB.misfit(FB.model(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a0 + e * da, b0 + e * db, scheme), q)
        errs.append(abs(Je - J0 - e * slope))
    assert abs(slope) > 0
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


@pytest.mark.parametrize("pz", range(5))
def test_hessian_column_is_difference_of_gradients(pz):
    """Scheme I makes J exactly quadratic in the contrasts, so grad J(m + e u_{b,j}) -
    grad J(m) = e H[:, (b, j)] for a unit vector u at node j in parameter b."""
    w = I.small_freq_case(seed=20 + pz, pz=pz, nx=7, nz=6, ns=2, nr=5, nf=3)
    fg = fgrid(w)
    q = FB.model(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, w.xi_a, w.xi_b, FB.NONLINEAR)
    a0, b0 = 0.5 * w.xi_a.astype(np.float64), 0.2 * w.xi_b.astype(np.float64)
    j = 17
    iz, ix = divmod(j, fg.nx)
    H = FB.hessian_column(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, j)
    _, ga0, gb0 = FB.gradient(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a0, b0, q, FB.LINEAR)
    e = 0.05
    for b in range(2):
        a1, b1 = a0.copy(), b0.copy()
        (a1 if b == 0 else b1)[iz, ix] += e
        _, ga1, gb1 = FB.gradient(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a1, b1, q, FB.LINEAR)
        np.testing.assert_allclose((ga1 - ga0) / e, H[0, b], rtol=1e-8, atol=1e-10 * np.abs(H).max())
        np.testing.assert_allclose((gb1 - gb0) / e, H[1, b], rtol=1e-8, atol=1e-10 * np.abs(H).max())


def test_reduced_hessian_cross_terms_paper_claim():
    """Point-scatterer analysis (Sec. "Point-scatterer Analysis"): with sources and receivers
    evenly around x_0, the cross-parameter term of the reduced Hessian vanishes for K-rho and
    1/K-1/rho and not for the other three; K-rho and 1/K-1/rho have the same reduced Hessian."""
    w = I.freq_paper(n=5, dx=5.0, nf=6, df=1.0)
    fg = fgrid(w)
    j = w.centre_index()
    H = {pz: FB.reduced_hessian(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, j) for pz in range(5)}
    for pz in range(5):
        np.testing.assert_allclose(H[pz], H[pz].T, rtol=1e-12)
        assert np.all(np.linalg.eigvalsh(H[pz]) > 0)
        c = abs(H[pz][0, 1]) / math.sqrt(H[pz][0, 0] * H[pz][1, 1])
        if pz in (3, 4):
            assert c < 1e-12, (pz, c)
        else:
            assert c > 0.1, (pz, c)
    np.testing.assert_allclose(H[3], H[4], rtol=1e-12)
