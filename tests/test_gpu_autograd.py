"""torch.autograd through the CUDA forward model: gradients of a torch-written misfit agree
with the oracle, pass a Taylor test at 6 step sizes, and do not depend on whether the
wavefield history is kept whole or checkpointed and recomputed."""
import numpy as np
import pytest

import oracle
from paper_1804_01184_gb300 import inputs as I
from tests._common import GRAD_TOL, gpu_grid, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import autograd, build
    build.build()
    return autograd


def setup(seed=80, pz=I.PZ_VP_RHO, nt=260):
    w = I.small_case(seed=seed, nx=58, nz=50, nt=nt, order=8, sponge=8, ns=3, nr=7, pz=pz)
    og = oracle_grid(w)
    data = oracle.model(og, pz, w.xi_a * 1.5, w.xi_b * 0.5, w.src_xy, w.wavelet, w.rec_xy).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return w, og, data, dev


def misfit(A, w, g, a, b, dev, data, budget=None):
    tr = A.model(a, b, g, w.pz, dev(w.src_xy), dev(w.wavelet), dev(w.rec_xy), budget)
    return 0.5 * ((tr.double() - dev(data).double()) ** 2).sum()


@pytest.mark.parametrize("pz", [I.PZ_VP_RHO, I.PZ_INVK_INVRHO])
def test_autograd_matches_oracle(A, pz):
    w, og, data, dev = setup(pz=pz)
    a = dev(w.xi_a * 0.5).requires_grad_()
    b = dev(w.xi_b * 0.5).requires_grad_()
    J = misfit(A, w, gpu_grid(w), a, b, dev, data)
    J.backward()
    J_ref, G_ref = oracle.gradient(og, pz, w.xi_a * 0.5, w.xi_b * 0.5, w.src_xy, w.wavelet, w.rec_xy, data)
    assert abs(J.item() - J_ref) <= 1e-4 * J_ref
    assert rel_l2(a.grad.cpu().numpy(), G_ref[pz, 0]) <= GRAD_TOL
    assert rel_l2(b.grad.cpu().numpy(), G_ref[pz, 1]) <= GRAD_TOL


def test_autograd_taylor_six_steps(A):
    w, og, data, dev = setup(seed=81, pz=I.PZ_IP_RHO)
    g = gpu_grid(w)
    a0 = dev(w.xi_a * 0.4).requires_grad_()
    b0 = dev(w.xi_b * 0.4).requires_grad_()
    J0 = misfit(A, w, g, a0, b0, dev, data)
    J0.backward()
    da, db = dev(I.random_like(w.xi_a.shape, 90, 0.05)), dev(I.random_like(w.xi_a.shape, 91, 0.05))
    lin = (a0.grad.double() * da.double()).sum() + (b0.grad.double() * db.double()).sum()
    hs = [0.2 / 2 ** k for k in range(6)]
    rem = []
    with torch.no_grad():
        for h in hs:
            Jh = misfit(A, w, g, a0 + h * da, b0 + h * db, dev, data)
            rem.append(abs((Jh - J0 - h * lin).item()))
    slopes = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    # FP32 traces: the remainder reaches the rounding floor at the smallest steps
    assert np.all(slopes[:3] > 1.7) and np.all(slopes[:3] < 2.3), slopes
    assert np.median(slopes) > 1.5, slopes


def test_checkpointed_history_gives_same_gradient(A):
    w, og, data, dev = setup(seed=82, pz=I.PZ_K_RHO, nt=300)
    g = gpu_grid(w)
    from paper_1804_01184_gb300 import fwi
    grads = []
    for budget in (1 << 36, fwi.fwi_workspace_bytes(g, w.ns, w.nr, fwi.OP_ADJOINT, 0)):
        a = dev(w.xi_a * 0.5).requires_grad_()
        b = dev(w.xi_b * 0.5).requires_grad_()
        misfit(A, w, g, a, b, dev, data, budget).backward()
        grads.append((a.grad.cpu().numpy(), b.grad.cpu().numpy()))
    for k in range(2):
        assert rel_l2(grads[1][k], grads[0][k]) <= 1e-6


def test_config_smooth_taylor_with_checkpoints(A):
    """Full differentiation workload: 1201 x 1201 (+40-cell sponge), 6000 steps, 16 shots,
    smooth random background + 4 anomalies; checkpoints every 200 steps with recomputation;
    Taylor test at 6 step sizes through torch.autograd."""
    from paper_1804_01184_gb300 import fwi
    w, (a_bg, b_bg) = I.config_smooth()
    g = gpu_grid(w)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    src, rec, wav = dev(w.src_xy), dev(w.rec_xy), dev(w.wavelet)
    data = fwi.fwi_model(g, w.pz, dev(w.xi_a), dev(w.xi_b), src, wav, rec)
    fwi.fwi_set_checkpoint(200)
    try:
        a0 = dev(a_bg).requires_grad_()
        b0 = dev(b_bg).requires_grad_()
        tr = A.model(a0, b0, g, w.pz, src, wav, rec)
        J0 = 0.5 * ((tr.double() - data.double()) ** 2).sum()
        J0.backward()
    finally:
        fwi.fwi_set_checkpoint(0)
    assert torch.isfinite(a0.grad).all() and torch.isfinite(b0.grad).all()
    da, db = dev(w.xi_a - a_bg), dev(w.xi_b - b_bg)          # towards the true model
    lin = (a0.grad.double() * da.double()).sum() + (b0.grad.double() * db.double()).sum()
    assert lin.item() < 0                                      # a descent direction
    rem = []
    with torch.no_grad():
        for h in [0.2 / 2 ** k for k in range(6)]:
            trh = fwi.fwi_model(g, w.pz, a0 + h * da, b0 + h * db, src, wav, rec)
            Jh = 0.5 * ((trh.double() - data.double()) ** 2).sum()
            rem.append(abs((Jh - J0 - h * lin).item()))
    slopes = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(slopes[:3] > 1.7) and np.all(slopes[:3] < 2.3), slopes
