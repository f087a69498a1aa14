"""fwi_model_noalloc: forward modelling for callers that cannot allocate device memory
(a service whose device memory is fixed at start-up, a plugin inside a framework that owns
all device memory, code where an allocation may block).  It runs on the library's built-in
scratch array instead of a caller workspace.  Two calls in a row, with different models,
must match the existing entry point fwi_model on a caller workspace -- bitwise, since both
run the same kernels on the same plan shape and shot grouping does not change a shot's
arithmetic; a problem too large for the built-in scratch must be refused with FWI_ENOMEM; a
bad contrast recorded in the scratch must be reported by fwi_status_noalloc.  This file is
collected last."""
import numpy as np
import pytest

from tests._common import TRACE_TOL, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, fwi
    build.build()
    return fwi


def test_noalloc_matches_fwi_model_on_two_calls(F):
    from paper_1804_01184_gb300 import inputs as I
    w = I.config_point(nt=500)               # 201 x 201 + 40-cell sponge, 8 shots, 64 receivers
    g = F.make_grid(**w.grid_kwargs())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    src, rec, wav = dev(w.src_xy), dev(w.rec_xy), dev(w.wavelet)
    models = [(dev(w.xi_a), dev(w.xi_b)), (dev(w.xi_a * 3.0), dev(w.xi_b * -2.0))]
    for xa, xb in models:                     # two calls in a row, each against fwi_model
        ref = F.fwi_model(g, w.pz, xa, xb, src, wav, rec).cpu().numpy()
        out = F.fwi_model_noalloc(g, w.pz, xa, xb, src, wav, rec)
        torch.cuda.synchronize()
        out = out.cpu().numpy()
        assert np.all(np.isfinite(out))
        np.testing.assert_array_equal(out, ref)
        assert rel_l2(out, ref) <= TRACE_TOL


def test_noalloc_refuses_problems_beyond_its_scratch(F):
    # 1481 x 1481 computational cells: ~9 MB per field, ~80 MB with one shot at a time
    g = F.make_grid(1401, 1401, 2.5, 2.5e-4, 100, order=8, sponge=40)
    need = F.fwi_workspace_bytes(g, 1, 1, F.OP_MODEL, 0)
    assert need > 64 << 20
    xa = torch.zeros((1401, 1401), dtype=torch.float32, device="cuda")
    xy = torch.tensor([[1500.0, 1500.0]], device="cuda")
    wav = torch.zeros(100, device="cuda")
    with pytest.raises(F.FwiError) as e:
        F.fwi_model_noalloc(g, 0, xa, xa, xy, wav, xy)
    assert e.value.code == -3 and "built-in scratch" in str(e.value)


def test_noalloc_reports_a_bad_contrast(F):
    """A contrast with 1 + xi <= 0 is a data-dependent error: the kernels record it in the
    built-in scratch, fwi_status_noalloc returns FWI_EINVAL and clears it, and the next good
    call reports nothing."""
    from paper_1804_01184_gb300 import inputs as I
    w = I.small_case(seed=90, nx=40, nz=36, nt=60, ns=2, nr=3)
    g = F.make_grid(**w.grid_kwargs())
    bad = w.xi_a.copy()
    bad[5, 7] = -1.0
    F.fwi_model_noalloc(g, w.pz, bad, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, check=False)
    with pytest.raises(F.FwiError) as e:
        F.fwi_status_noalloc()
    assert e.value.code == -1
    F.fwi_status_noalloc()                     # cleared
    with pytest.raises(F.FwiError) as e:       # check=True raises it directly
        F.fwi_model_noalloc(g, w.pz, bad, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    assert e.value.code == -1
    out = F.fwi_model_noalloc(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    assert torch.isfinite(out).all()
