"""CPU checks of the host-side pieces around the library: the seeded scatterers of Table
"tab:param_scat", the contrast grids and shape fit of the error bowls, the aperture weights,
and the steepest-descent loop (on a fake back end with a known quadratic misfit)."""
import numpy as np

from paper_1804_01184_gb300 import bowls as B
from paper_1804_01184_gb300 import inputs as I


def test_unknown_shape_scatterers():
    g = I.gaussian(41, 41, 5.0, (100.0, 100.0), 50.0)
    a, b = B.unknown_contrasts(g, "vp")
    assert np.allclose(a, 0.2 * g) and not b.any()
    a, b = B.unknown_contrasts(g, "rho")
    assert np.allclose(b, 0.2 * g) and not a.any()
    a, b = B.unknown_contrasts(g, "nonK")                     # (vii): no bulk-modulus contrast
    K = (1.0 + b.astype(np.float64)) * (1.0 + a.astype(np.float64)) ** 2
    assert np.abs(K - 1.0).max() < 1e-6 and a.max() > 0.19 and b.min() < -0.3
    w = B.unknown_scatterer("vii", nt=10)
    assert w.xi_a.shape == (w.nz, w.nx) and abs(w.xi_a.max() - 0.2) < 1e-3


def test_grid_around_holds_the_truth_and_zero():
    for t in (0.2, -0.3056, 0.0, 0.44):
        g = B.grid_around(t, 21)
        assert len(g) == 21 and np.min(np.abs(g - t)) < 1e-12
        assert g[0] <= min(0.0, t) and g[-1] >= max(0.0, t)
        assert np.allclose(np.diff(g), np.diff(g)[0])


def test_true_point_inverts_the_parameterization_definitions():
    """Table 1 contrasts of vp = 1.2, rho = 0.9 (relative to the reference) in each
    parameterization, checked against the definitions Ip = rho vp and K = rho vp^2."""
    v, r = 1.2, 0.9
    assert np.allclose(B.true_point(I.PZ_VP_RHO, v - 1, r - 1), (v - 1, r - 1))
    assert np.allclose(B.true_point(I.PZ_IP_RHO, v - 1, r - 1), (r * v - 1, r - 1))
    assert np.allclose(B.true_point(I.PZ_VP_IP, v - 1, r - 1), (v - 1, r * v - 1))
    assert np.allclose(B.true_point(I.PZ_K_RHO, v - 1, r - 1), (r * v * v - 1, r - 1))
    assert np.allclose(B.true_point(I.PZ_INVK_INVRHO, v - 1, r - 1), (1 / (r * v * v) - 1, 1 / r - 1))


def test_bowl_shape_of_a_known_quadratic():
    """A quadratic bowl with curvatures 1 and 16 whose long axis lies at 30 degrees."""
    a = np.linspace(-1, 1, 21)
    b = np.linspace(-1, 1, 21)
    th = np.radians(30.0)
    u = np.array([np.cos(th), np.sin(th)])
    v = np.array([-np.sin(th), np.cos(th)])
    A, Bm = np.meshgrid(a, b, indexing="ij")
    P = np.stack([A - 0.1, Bm + 0.2], axis=-1)
    J = 0.5 * (1.0 * (P @ u) ** 2 + 16.0 * (P @ v) ** 2)
    s = B.bowl_shape(J, a, b, half=3)
    assert abs(s["condition"] - 16.0) < 1e-6
    assert abs(s["angle_deg"] - 30.0) < 1e-6
    assert abs(s["argmin"][0] - 0.1) < 1e-12 and abs(s["argmin"][1] + 0.2) < 1e-12


def test_aperture_weights_select_scattering_angles():
    src = np.array([[0.0, -100.0]])
    rec = np.array([[0.0, 100.0], [100.0, 0.0], [0.0, -90.0]])      # 0, 90, 180 degrees at x0 = 0
    w = B.aperture_weights(src, rec, (0.0, 0.0), 0.0, 90.0)
    np.testing.assert_array_equal(w, [[1.0, 1.0, 0.0]])
    w = B.aperture_weights(src, rec, (0.0, 0.0), 135.0, 180.0)
    np.testing.assert_array_equal(w, [[0.0, 0.0, 1.0]])


def test_steepest_descent_loop_on_a_quadratic():
    """The shared descent loop (line search over 8 trial steps, re-centred step) on a fake back
    end with a known 2-parameter quadratic misfit: monotone, and converges to the minimum."""
    from paper_1804_01184_gb300 import invert as V
    H = np.array([[3.0, 1.0], [1.0, 2.0]])
    m_star = np.array([0.3, -0.2])

    class Quad(V._SteepestDescent):
        def __init__(self):
            self.g = object()          # a known shape: the parameters are two scalars
            self.alpha = None

        def misfit(self, m):
            d = np.array(m, float) - m_star
            return 0.5 * d @ H @ d

        def gradient(self, m):
            d = np.array(m, float) - m_star
            return self.misfit(m), tuple(H @ d)

        def misfits(self, models):
            return np.array([self.misfit(m) for m in models])

    m, hist = Quad().run((0.0, 0.0), iters=40)
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert np.hypot(m[0] - m_star[0], m[1] - m_star[1]) < 1e-4


def test_scattering_angles_and_pattern_summary():
    from paper_1804_01184_gb300 import patterns as PT
    src = np.array([[0.0, -100.0]])
    th = np.radians(np.arange(0.0, 360.0, 5.0))
    rec = np.stack([100.0 * np.sin(th), 100.0 * np.cos(th)], axis=1)   # angle from the +z axis
    ang = PT.scattering_angles(src, rec, (0.0, 0.0))
    expect = np.degrees(np.arccos(np.clip(np.cos(th), -1, 1)))
    np.testing.assert_allclose(ang[0], expect, atol=1e-9)
    e = PT.cos2(ang)
    s = PT.pattern_summary(e, ang)
    assert s["0"] == 1.0 and s["180"] == 1.0 and s["90"] < 1e-12 and abs(s["45"] - 0.5) < 1e-4
