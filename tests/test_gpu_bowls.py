"""Error bowls (Sec. "Error-bowl Analysis") through the batching engine: the misfit surface of
a scatterer of known shape over a grid of its two contrasts.  The bowl is exactly zero at the
true contrasts (same discrete model), its values match the FP64 oracle within the bound the
trace tolerance implies, and fwi_misfit agrees with a float64 reduction."""
import numpy as np
import pytest

import oracle
from paper_1804_01184_gb300 import inputs as I
from tests._common import GRAD_TOL, TRACE_TOL, gpu_grid, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import bowls, build, fwi
    build.build()
    return fwi, bowls


def test_misfit_kernel_matches_float64(L):
    F, _ = L
    a = I.random_like((3, 17, 333), 1, 1.0)
    b = I.random_like((3, 17, 333), 2, 1.0)
    J = F.fwi_misfit(a, b).item()
    ref = 0.5 * np.sum((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    assert abs(J - ref) <= 1e-12 * ref


@pytest.mark.parametrize("pz", [I.PZ_K_RHO, I.PZ_VP_IP])
def test_bowl_zero_at_truth_and_oracle_values(L, pz):
    F, B = L
    w = I.small_case(seed=31, nx=50, nz=46, nt=160, order=8, sponge=6, ns=3, nr=8, pz=pz)
    g = I.gaussian(w.nx, w.nz, w.dx, I.centre_of(w.nx, w.nz, w.dx), 15.0)
    ga = np.array([-0.1, 0.0, 0.1, 0.2, 0.3], np.float32)
    gb = np.array([-0.2, -0.1, 0.0, 0.1], np.float32)
    ta, tb = 3, 1                                          # truth (0.2, -0.1)
    w.xi_a, w.xi_b = g * ga[ta], g * gb[tb]
    data = F.fwi_model(gpu_grid(w), pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    J, launches = B.error_bowl(w, g, pz, data, ga, gb, arena_bytes=1 << 30)
    assert launches > 0
    assert J[ta, tb] == 0.0 and np.unravel_index(int(np.argmin(J)), J.shape) == (ta, tb)
    og = oracle_grid(w)
    d_ref = oracle.model(og, pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    eb = 2 * TRACE_TOL * np.linalg.norm(d_ref)             # trace error of both sides
    for ia, ib in [(0, 0), (4, 3), (1, 2), (3, 0)]:
        tr = oracle.model(og, pz, g * ga[ia], g * gb[ib], w.src_xy, w.wavelet, w.rec_xy)
        r = np.linalg.norm(tr - d_ref)
        J_ref = 0.5 * r * r
        assert abs(J[ia, ib] - J_ref) <= r * eb + 0.5 * eb * eb, (ia, ib, J[ia, ib], J_ref)
    s = B.bowl_shape(J, ga, gb, half=1)
    assert s["argmin"] == (float(ga[ta]), float(gb[tb])) and s["condition"] >= 1.0


def test_weighted_gradient_is_the_adjoint_of_the_masked_residual(L):
    """fwi_gradient_weighted with 0/1 aperture weights equals fwi_adjoint given the masked
    residual w (d_mod - data) bitwise, its misfit equals the masked sum, and all-one weights
    reproduce fwi_gradient bitwise."""
    F, B = L
    w = I.small_case(seed=33, nx=48, nz=44, nt=140, order=8, sponge=6, ns=3, nr=10)
    c = I.centre_of(w.nx, w.nz, w.dx)
    w.src_xy, w.rec_xy = I.circle(w.ns, 90.0, c), I.circle(w.nr, 90.0, c, 0.5)
    g = gpu_grid(w)
    wt = B.aperture_weights(w.src_xy, w.rec_xy, c, 0.0, 90.0)
    assert 0 < wt.sum() < wt.size
    data = I.random_like((w.ns, w.nr, w.nt), 9, 1e3)
    a0, b0 = w.xi_a * 0.5, w.xi_b * 0.5
    J, G = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data, weights=wt)
    tr = F.fwi_model(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy)
    wd, dd = torch.from_numpy(wt).cuda()[:, :, None], torch.from_numpy(data).cuda()
    res = (tr - dd) * wd
    G2 = F.fwi_adjoint(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, res)
    assert torch.equal(G, G2)
    r64 = (tr.double() - dd.double()) ** 2 * wd.double()
    assert abs(J.item() - 0.5 * r64.sum().item()) <= 1e-9 * J.item()
    Jm = F.fwi_misfit(tr, dd, weights=wt, nt=w.nt).item()
    assert abs(Jm - J.item()) <= 1e-9 * J.item()
    J1, G1 = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data, weights=np.ones_like(wt))
    J0, G0 = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
    assert torch.equal(G1, G0) and J1.item() == J0.item()


@pytest.mark.parametrize("lo,hi", [(0.0, 90.0), (135.0, 180.0)])
def test_weighted_gradient_matches_the_oracle(L, lo, hi):
    """Limited aperture (Sec. "Hierarchical Inversion"): fwi_gradient_weighted with the 0/1
    weights of a scattering-angle range against the oracle -- the gradient is oracle.adjoint
    of the masked residual w (oracle.model - data), the misfit 1/2 sum w (oracle.model -
    data)^2 -- at the gradient and trace tolerances, for every field of all five
    parameterizations."""
    F, B = L
    w = I.small_case(seed=34, nx=52, nz=48, nt=180, order=8, sponge=6, ns=4, nr=16, pz=I.PZ_VP_RHO)
    c = I.centre_of(w.nx, w.nz, w.dx)
    w.src_xy, w.rec_xy = I.circle(w.ns, 95.0, c), I.circle(w.nr, 95.0, c, 0.5)
    wt = B.aperture_weights(w.src_xy, w.rec_xy, c, lo, hi)
    assert 0 < wt.sum() < wt.size
    og = oracle_grid(w)
    data = oracle.model(og, w.pz, w.xi_a * 1.4, w.xi_b * 0.6, w.src_xy, w.wavelet, w.rec_xy).astype(np.float32)
    a0, b0 = (w.xi_a * 0.5).astype(np.float32), (w.xi_b * 0.5).astype(np.float32)
    d_mod = oracle.model(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy)
    r = d_mod - data.astype(np.float64)
    G_ref = oracle.adjoint(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, wt[:, :, None] * r)
    J_ref = 0.5 * float(np.sum(wt[:, :, None] * r * r))
    J, G = F.fwi_gradient(gpu_grid(w), w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data, weights=wt)
    G = G.cpu().numpy()
    assert abs(J.item() - J_ref) <= TRACE_TOL * J_ref
    for pz in range(5):
        for k in range(2):
            assert rel_l2(G[pz, k], G_ref[pz, k]) <= GRAD_TOL, (pz, k, rel_l2(G[pz, k], G_ref[pz, k]))
