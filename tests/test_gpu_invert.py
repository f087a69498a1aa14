"""Steepest-descent inversion with an engine-batched line search: the misfit decreases at every
accepted iteration, a known-shape point scatterer's contrasts move towards the truth, and an
unknown-shape inversion lowers the misfit too."""
import numpy as np
import pytest

from paper_1804_01184_gb300 import inputs as I
from tests._common import gpu_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, fwi, invert
    build.build()
    return fwi, invert


def setup(F, seed, pz, shape_kind="gaussian"):
    w = I.small_case(seed=seed, nx=56, nz=52, nt=220, order=8, sponge=8, ns=4, nr=12, pz=pz, f_peak=20.0)
    c = I.centre_of(w.nx, w.nz, w.dx)
    w.src_xy = I.circle(w.ns, 100.0, c)
    w.rec_xy = I.circle(w.nr, 100.0, c, 0.5)
    g = I.gaussian(w.nx, w.nz, w.dx, c, 12.0) if shape_kind == "gaussian" else I.point(w.nx, w.nz)
    return w, g


@pytest.mark.parametrize("pz", [I.PZ_K_RHO, I.PZ_VP_RHO])
def test_known_shape_converges_towards_truth(L, pz):
    F, V = L
    w, g = setup(F, 41, pz)
    truth = (0.15, -0.1)
    data = F.fwi_model(gpu_grid(w), pz, g * np.float32(truth[0]), g * np.float32(truth[1]), w.src_xy, w.wavelet,
                       w.rec_xy)
    inv = V.Inversion(w, pz, data, shape=g)
    m, hist = inv.run((0.0, 0.0), iters=8)
    inv.close()
    assert len(hist) >= 5
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.1 * hist[0]
    err0 = np.hypot(*truth)
    assert np.hypot(m[0] - truth[0], m[1] - truth[1]) < 0.5 * err0


def test_unknown_shape_lowers_the_misfit(L):
    F, V = L
    w, g = setup(F, 42, I.PZ_VP_RHO)
    data = F.fwi_model(gpu_grid(w), I.PZ_VP_RHO, g * np.float32(0.2), g * np.float32(0.0), w.src_xy, w.wavelet,
                       w.rec_xy)
    z = torch.zeros((w.nz, w.nx), dtype=torch.float32, device="cuda")
    inv = V.Inversion(w, I.PZ_VP_RHO, data)
    m, hist = inv.run((z, z.clone()), iters=4)
    inv.close()
    assert all(b < a for a, b in zip(hist, hist[1:])) and hist[-1] < 0.9 * hist[0]   # plain steepest descent: slow
    assert torch.isfinite(m[0]).all() and torch.isfinite(m[1]).all()
