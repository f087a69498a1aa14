"""Frequency-domain Born modelling of Schemes I/II through the C ABI against the FP64 oracle
(oracle/fborn.py): Green tables and Born data for every parameterization and both maps,
the misfit and its gradient, the Scheme I Hessian column and reduced Hessian; tile edges
(ragged node chunks, more than 16 sources, more than 128 receivers); the paper's full
acquisition on sampled outputs; determinism and argument errors."""
import math

import numpy as np
import pytest

from oracle import fborn as FB
from paper_1804_01184_gb300 import inputs as I
from tests._common import GRAD_TOL, TRACE_TOL, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HESS_TOL = 1e-4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, fborn
    build.build()
    return fborn


def ofg(w):
    return FB.FGrid(**w.fgrid_kwargs())


def crel(a, b):
    """Relative L2 distance of complex arrays."""
    a, b = np.asarray(a, np.complex128), np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_data(w, pz, a, b, scheme, incident=True):
    return FB.model(ofg(w), w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a, b, scheme, with_incident=incident)


CASES = [dict(seed=0), dict(seed=5, nx=9, nz=7, ns=17, nr=130, nf=2)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("pz", range(5))
def test_born_data_matches_oracle(B, case, scheme, pz):
    w = I.small_freq_case(pz=pz, **case)
    acq = B.acquisition(w)
    for incident in (True, False):
        d = acq.model(pz, w.xi_a, w.xi_b, scheme=scheme, incident=incident).cpu().numpy()
        ref = oracle_data(w, pz, w.xi_a, w.xi_b, scheme, incident)
        assert crel(d, ref) <= TRACE_TOL


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("pz", range(5))
def test_gradient_matches_oracle(B, case, scheme, pz):
    w = I.small_freq_case(pz=pz, **case)
    acq = B.acquisition(w)
    q = oracle_data(w, pz, 1.4 * w.xi_a, 0.6 * w.xi_b, 2).astype(np.complex64)
    a0, b0 = 0.5 * w.xi_a, -0.3 * w.xi_b
    J, G = acq.gradient(pz, a0, b0, q, scheme=scheme)
    Jr, ga, gb = FB.gradient(ofg(w), w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, a0, b0,
                             q.astype(np.complex128), scheme)
    assert abs(J.item() - Jr) <= 1e-5 * Jr
    G = G.cpu().numpy()
    assert rel_l2(G[0], ga) <= GRAD_TOL
    assert rel_l2(G[1], gb) <= GRAD_TOL


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("pz", range(5))
def test_hessian_column_matches_oracle(B, case, pz):
    w = I.small_freq_case(pz=pz, **case)
    acq = B.acquisition(w)
    jx, jz = w.nx // 3, w.nz // 2
    H = acq.hessian(pz, jx, jz).cpu().numpy()
    ref = FB.hessian_column(ofg(w), w.freqs, w.spectrum, w.src_xy, w.rec_xy, pz, jz * w.nx + jx)
    assert rel_l2(H, ref) <= HESS_TOL
    for a in range(2):
        for b in range(2):
            assert rel_l2(H[a, b], ref[a, b]) <= 10 * HESS_TOL


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("scheme", [1, 2])
def test_gradient_hessian_in_one_pass(B, case, scheme):
    """fwi_fborn_gradient_hessian gives what fwi_fborn_gradient and fwi_fborn_hessian give
    separately (the same sums in the same order, bitwise), and its Hessian matches the oracle;
    with 17 sources (two source blocks) and 130 receivers (two residual tiles)."""
    w = I.small_freq_case(**case)
    acq = B.acquisition(w)
    a0, b0 = 0.5 * w.xi_a, -0.3 * w.xi_b
    q = acq.model(1, w.xi_a, w.xi_b, scheme=2).cpu().numpy()
    jx, jz = w.nx // 3, w.nz // 2
    for pz in (0, 2, 4):
        J, G = acq.gradient(pz, a0, b0, q, scheme=scheme)
        H = acq.hessian(pz, jx, jz)
        J2, G2, H2 = acq.gradient_hessian(pz, a0, b0, q, jx, jz, scheme=scheme)
        assert torch.equal(J, J2) and torch.equal(G, G2) and torch.equal(H, H2)
    ref = FB.hessian_column(ofg(w), w.freqs, w.spectrum, w.src_xy, w.rec_xy, 4, jz * w.nx + jx)
    assert rel_l2(H2.cpu().numpy(), ref) <= HESS_TOL
    acq.status()


def test_reduced_hessian_cross_terms_paper_claim(B):
    """With sources and receivers evenly around x_0 the K-rho and 1/K-1/rho reduced Hessians
    have no cross-parameter term (to FP32 rounding); vp-rho, Ip-rho and vp-Ip do."""
    w = I.freq_paper(n=21, nf=12, df=1.0)
    acq = B.acquisition(w)
    c = w.nx // 2
    for pz in range(5):
        H = acq.reduced_hessian(pz, c, c).cpu().numpy()
        x = abs(H[0, 1]) / math.sqrt(H[0, 0] * H[1, 1])
        assert abs(H[0, 1] - H[1, 0]) <= 1e-5 * abs(H).max()
        assert (x < 1e-5) if pz in (3, 4) else (x > 0.1), (pz, x)


def test_paper_acquisition_sampled(B):
    """The benchmark's configuration (121 x 121 nodes, 60 frequencies, 10 sources, 100
    receivers): data entries of a few (source, receiver) pairs at all frequencies against the
    oracle run on those pairs alone; the gradient's directional derivative against a central
    difference of GPU misfits (exact for the quadratic Scheme I misfit); the Hessian column at
    x_0 against the oracle on two of the frequencies."""
    w = I.freq_paper()
    acq = B.acquisition(w)
    d = acq.model(0, w.xi_a, w.xi_b, scheme=2).cpu().numpy()
    ss, rr = [0, 3, 7], [0, 41, 99]
    ref = FB.model(ofg(w), w.freqs, w.spectrum, w.src_xy[ss], w.rec_xy[rr], 0, w.xi_a, w.xi_b, 2)
    got = d[:, ss][:, :, rr]
    assert crel(got, ref) <= TRACE_TOL
    # gradient along a direction, Scheme I (quadratic misfit)
    q = acq.model(0, w.xi_a, w.xi_b, scheme=2)
    a0 = np.zeros_like(w.xi_a)
    _, G = acq.gradient(0, a0, a0, q, scheme=1)
    G = G.cpu().numpy()
    da = I.gaussian(w.nx, w.nz, w.dx, ((w.nx - 1) / 2 * w.dx, (w.nz - 1) / 2 * w.dx), 40.0)
    db = 0.5 * da
    eps = 0.05
    Jp = acq.gradient(0, eps * da, eps * db, q, scheme=1)[0].item()
    Jm = acq.gradient(0, -eps * da, -eps * db, q, scheme=1)[0].item()
    slope = float(np.sum(G[0] * da) + np.sum(G[1] * db))
    assert abs((Jp - Jm) / (2 * eps) - slope) <= 1e-3 * abs(slope)
    # Hessian column at x_0 on two frequencies
    sub = [9, 29]
    w2 = I.freq_paper()
    w2.freqs, w2.spectrum = w.freqs[sub], w.spectrum[sub]
    acq2 = B.acquisition(w2)
    c = w.nx // 2
    H = acq2.hessian(3, c, c).cpu().numpy()
    ref = FB.hessian_column(ofg(w2), w2.freqs, w2.spectrum, w2.src_xy, w2.rec_xy, 3, c * w.nx + c)
    assert rel_l2(H, ref) <= HESS_TOL


def test_deterministic_and_errors(B):
    from paper_1804_01184_gb300 import fwi as F
    w = I.small_freq_case(seed=7)
    acq = B.acquisition(w)
    d1 = acq.model(1, w.xi_a, w.xi_b).cpu().numpy()
    d2 = acq.model(1, w.xi_a, w.xi_b).cpu().numpy()
    np.testing.assert_array_equal(d1, d2)
    _, g1 = acq.gradient(2, w.xi_a, w.xi_b, d1 * 0.9)
    _, g2 = acq.gradient(2, w.xi_a, w.xi_b, d1 * 0.9)
    np.testing.assert_array_equal(g1.cpu().numpy(), g2.cpu().numpy())
    acq.status()                                          # no bounded wait of the contraction expired
    fg = B.make_fgrid(w.nx, w.nz, w.nf, w.dx, w.x0, w.z0)
    on_node = w.src_xy.copy()
    on_node[0] = (w.x0 + 2 * w.dx, w.z0 + 3 * w.dx)
    with pytest.raises(F.FwiError):
        B.Acquisition(fg, w.freqs, w.spectrum, on_node, w.rec_xy)
    bad_f = w.freqs.copy()
    bad_f[1] = 0.0
    with pytest.raises(F.FwiError):
        B.Acquisition(fg, bad_f, w.spectrum, w.src_xy, w.rec_xy)
    with pytest.raises(F.FwiError):
        acq.hessian(0, w.nx, 0)
    with pytest.raises(F.FwiError):
        acq.model(0, w.xi_a, w.xi_b, scheme=3)
    with pytest.raises(F.FwiError):
        acq.gradient_hessian(0, w.xi_a, w.xi_b, d1, w.nx, 0)           # node off the grid
    # the Hessian terms keep u_p(x_j) of every point in shared memory: at most 2048 points
    big = I.small_freq_case(seed=8, nx=3, nz=3, ns=1000, nr=1049, nf=1)
    ab = B.acquisition(big)
    qb = np.zeros((1, big.ns, big.nr), np.complex64)
    for call in (lambda: ab.hessian(0, 1, 1), lambda: ab.gradient_hessian(0, big.xi_a, big.xi_b, qb, 1, 1)):
        with pytest.raises(F.FwiError):
            call()
    acq.status()


def test_born_inversions_converge(B):
    """Steepest descent on the frequency-domain Born misfit of a known-shape Gaussian scatterer
    whose true contrasts the inversion can represent -- (-0.3, 0.1) g in 1/K-1/rho under
    Scheme I (the linear map is exact there) and (0.2, 0) g in vp-rho under Scheme II (exact
    map) -- reaches them; every accepted iteration lowers the misfit."""
    from paper_1804_01184_gb300 import invert as V
    w = I.freq_paper(n=41, nf=20, df=0.5)
    c = (w.nx - 1) / 2 * w.dx
    g = I.gaussian(w.nx, w.nz, w.dx, (c, c), 50.0)
    acq = B.acquisition(w)
    for pz, scheme, truth in ((4, 1, (-0.3, 0.1)), (0, 2, (0.2, 0.0))):
        data = acq.model(pz, np.float32(truth[0]) * g, np.float32(truth[1]) * g, scheme=2)
        inv = V.BornInversion(acq, pz, data, scheme, shape=g)
        m, hist = inv.run((0.0, 0.0), iters=12)
        assert all(b < a for a, b in zip(hist, hist[1:]))
        assert hist[-1] < 1e-3 * hist[0], (pz, hist)
        assert np.hypot(m[0] - truth[0], m[1] - truth[1]) < 0.01, (pz, m)


def test_degenerate_cases(B):
    """Zero contrasts leave only the direct field (the scattered part is exactly zero); at the
    model that generated the data the residual is the data's FP32 rounding alone, so the misfit
    and the gradient vanish to that level; a single node, source and receiver work."""
    w = I.small_freq_case(seed=11)
    acq = B.acquisition(w)
    z = np.zeros_like(w.xi_a)
    assert not acq.model(2, z, z, incident=False).abs().max().item()
    direct = acq.model(2, z, z).cpu().numpy()
    ref = FB.model(ofg(w), w.freqs, w.spectrum, w.src_xy, w.rec_xy, 2, z, z, 2)
    assert crel(direct, ref) <= TRACE_TOL
    for scheme in (1, 2):
        q = acq.model(3, w.xi_a, w.xi_b, scheme=scheme)
        J, G = acq.gradient(3, w.xi_a, w.xi_b, q, scheme=scheme)
        J1, G1 = acq.gradient(3, 0.9 * w.xi_a, 0.9 * w.xi_b, q, scheme=scheme)
        assert J.item() <= 1e-10 * 0.5 * (q.abs() ** 2).sum().item()
        assert G.abs().max().item() <= 1e-4 * G1.abs().max().item()
    one = I.small_freq_case(seed=12, nx=1, nz=1, ns=1, nr=1, nf=1)
    a1 = B.acquisition(one)
    d = a1.model(0, one.xi_a, one.xi_b, scheme=2).cpu().numpy()
    ref = FB.model(ofg(one), one.freqs, one.spectrum, one.src_xy, one.rec_xy, 0, one.xi_a, one.xi_b, 2)
    assert crel(d, ref) <= TRACE_TOL
    H = a1.hessian(4, 0, 0).cpu().numpy()
    refH = FB.hessian_column(ofg(one), one.freqs, one.spectrum, one.src_xy, one.rec_xy, 4, 0)
    assert rel_l2(H, refH) <= HESS_TOL


@pytest.mark.parametrize("rho_o, vp_o, amp", [(1.0, 1500.0, 0.15), (2.5e6, 4000.0, 0.15), (2000.0, 2000.0, 1e-6),
                                           (2000.0, 2000.0, 0.9)])
def test_row_scaling_over_magnitudes(B, rho_o, vp_o, amp):
    """The tensor-core data contraction scales each operand row by a power of two taken from
    the tables' and the contrasts' largest values before its FP16 split: Born data for
    reference media and contrast amplitudes spanning many decades (table values from ~0.1 to
    ~1e6, contrasts from 1e-6 to ~1e3 under the exact map) match the oracle to the same
    tolerance, and no bounded wait expires."""
    import dataclasses
    w = dataclasses.replace(I.small_freq_case(seed=21, nx=17, nz=13, ns=5, nr=40, nf=3, amp=amp), rho_o=rho_o,
                            vp_o=vp_o)
    acq = B.acquisition(w)
    for scheme in (1, 2):
        d = acq.model(0, w.xi_a, w.xi_b, scheme=scheme, incident=False).cpu().numpy()
        ref = oracle_data(w, 0, w.xi_a, w.xi_b, scheme, incident=False)
        assert np.isfinite(d).all()
        assert crel(d, ref) <= TRACE_TOL
    acq.status()


def test_diffraction_patterns(B):
    """Sec. "Diffraction-pattern Analysis": a unit point contrast at x_0 with sources and
    receivers on a circle around it scatters the same energy at every angle for 1/K (and K, and
    vp in vp-rho, whose maps keep only the bulk-modulus term) and as cos^2 of the scattering
    angle for 1/rho (and rho in K-rho); the patterns do not depend on the sign of the map."""
    from paper_1804_01184_gb300 import patterns as PT
    w = I.freq_paper(n=21, nf=8, df=1.0)
    acq = B.acquisition(w)
    c = w.nx // 2
    ang = PT.scattering_angles(w.src_xy, w.rec_xy, (0.0, 0.0))
    for pz, param in ((4, 0), (3, 0), (0, 0)):
        e = PT.diffraction_pattern(acq, pz, param, c, c)
        assert e.std() <= 1e-5 * e.mean(), (pz, param)
    for pz in (4, 3):
        e = PT.diffraction_pattern(acq, pz, 1, c, c)
        np.testing.assert_allclose(e / e.max(), PT.cos2(ang) / PT.cos2(ang).max(), atol=2e-5)
    s = PT.pattern_summary(PT.diffraction_pattern(acq, 4, 1, c, c), ang)
    assert s["90"] < 0.01 and s["0"] > 0.98 and s["180"] > 0.98


def test_born_error_bowl_vanishes_at_truth(B):
    """Scheme II error bowl of a Gaussian vp scatterer in vp-rho: the contrast grid holds the
    truth (0.2, 0), where the misfit falls to the data's rounding level, and it is the bowl's
    minimum; every other point is far above it."""
    from paper_1804_01184_gb300 import bowls as BW
    w = I.freq_paper(n=31, nf=10, df=1.0)
    h = (w.nx - 1) / 2 * w.dx
    g = I.gaussian(w.nx, w.nz, w.dx, (h, h), 50.0)
    acq = B.acquisition(w)
    data = acq.model(0, np.float32(0.2) * g, 0 * g, scheme=2)
    ga, gb = BW.grid_around(0.2, 7), BW.grid_around(0.0, 7)
    J = BW.born_error_bowl(acq, g, 0, data, ga, gb, 2)
    ia, ib = np.unravel_index(np.argmin(J), J.shape)
    assert abs(ga[ia] - 0.2) < 1e-12 and abs(gb[ib]) < 1e-12
    rest = np.delete(J.ravel(), np.argmin(J))
    assert J.min() <= 1e-8 * rest.min()
