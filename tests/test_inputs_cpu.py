"""CPU checks of the seeded scatterers of Table "tab:param_scat" that the inversions use."""
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
