"""Steepest-descent inversion with an engine-batched line search: the misfit decreases at every
accepted iteration, a known-shape point scatterer's contrasts move towards the truth, and an
unknown-shape inversion lowers the misfit too."""
import numpy as np
import pytest

from paper_1804_01184_gb300 import inputs as I
from tests._common import GRAD_TOL, gpu_grid, oracle_grid

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


def oracle_descent(V, w, pz, data, shape):
    """The same steepest-descent loop as invert.Inversion (its line search, step rule and
    projection on the known shape), driven by the FP64 oracle: the gradient from
    oracle.gradient, the trial misfits from oracle.model."""
    import oracle
    og = oracle_grid(w)
    d64 = np.asarray(data, np.float64)

    class Descent(V._SteepestDescent):
        def __init__(self):
            self.alpha = None
            self.g = np.asarray(shape, np.float32)

        def fields(self, m):
            return self.g * np.float32(m[0]), self.g * np.float32(m[1])

        def gradient(self, m):
            xa, xb = self.fields(m)
            J, G = oracle.gradient(og, pz, xa, xb, w.src_xy, w.wavelet, w.rec_xy, d64)
            g64 = self.g.astype(np.float64)
            return J, (float(np.sum(G[pz, 0] * g64)), float(np.sum(G[pz, 1] * g64)))

        def misfits(self, models):
            out = []
            for m in models:
                xa, xb = self.fields(m)
                r = oracle.model(og, pz, xa, xb, w.src_xy, w.wavelet, w.rec_xy) - d64
                out.append(0.5 * float(np.sum(r * r)))
            return np.array(out)

    return Descent()


@pytest.mark.parametrize("pz", [I.PZ_K_RHO, I.PZ_IP_RHO])
def test_known_shape_iterates_match_the_oracle_loop(L, pz):
    """Three iterations of invert.Inversion (Scheme III, engine-batched line search) against
    the same loop driven by oracle gradients and misfits: the misfit histories agree to the
    trace tolerance's bound on J and the iterates to the gradient tolerance."""
    F, V = L
    import oracle
    w, g = setup(F, 43, pz)
    truth = (0.15, -0.1)
    data = oracle.model(oracle_grid(w), pz, g * np.float32(truth[0]), g * np.float32(truth[1]), w.src_xy,
                        w.wavelet, w.rec_xy).astype(np.float32)
    inv = V.Inversion(w, pz, data, shape=g)
    m, hist = inv.run((0.0, 0.0), iters=3)
    inv.close()
    ref = oracle_descent(V, w, pz, data, g)
    m_ref, hist_ref = ref.run((0.0, 0.0), iters=3)
    assert len(hist) == len(hist_ref) == 4
    for J, Jr in zip(hist, hist_ref):
        assert abs(J - Jr) <= 1e-3 * Jr, (hist, hist_ref)
    for k in range(2):
        assert abs(m[k] - m_ref[k]) <= GRAD_TOL * np.hypot(*m_ref), (m, m_ref)
