"""The bounds-checked debug build (libfwi_checked.so, -DFWI_CHECKED): every global load and
store of the time-step kernels tests its offset against its field and records a failure in
the operation's status word instead of trapping (the substitute for a memory checker, which
is not available here).  On the parity cases -- narrow and multi-strip grids, orders 4 and 8,
with and without sponge, checkpointed gradients -- it must report nothing and give results
bitwise equal to the default build's, which also ties the default build's accesses to the
checked ones."""
import numpy as np
import pytest

from paper_1804_01184_gb300 import inputs as I
from tests._common import gpu_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    dict(seed=11, nx=75, nz=53, nt=120, order=8, sponge=10, ns=3, nr=9, pz=I.PZ_VP_RHO),
    dict(seed=12, nx=61, nz=70, nt=100, order=4, sponge=7, ns=2, nr=5, pz=I.PZ_IP_RHO),
    dict(seed=13, nx=40, nz=33, nt=90, order=8, sponge=0, ns=2, nr=4, pz=I.PZ_VP_IP),
    dict(seed=71, nx=231, nz=38, nt=80, order=8, sponge=5, ns=3, nr=5, pz=I.PZ_K_RHO),
    dict(seed=72, nx=150, nz=47, nt=70, order=4, sponge=9, ns=2, nr=6, pz=I.PZ_INVK_INVRHO),
]


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, fwi
    build.build(checked=True)
    return fwi


def run_all(F, w):
    g = gpu_grid(w)
    da, db = I.random_like(w.xi_a.shape, w.nx, 0.05), I.random_like(w.xi_a.shape, w.nz, 0.05)
    data = I.random_like((w.ns, w.nr, w.nt), 3, 1e3)
    out = [F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy),
           F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy),
           *F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)]
    try:
        F.fwi_set_checkpoint(max(1, w.nt // 3))
        out += list(F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data,
                                   work=F.workspace(g, w.ns, w.nr, F.OP_GRADIENT, 0)))
    finally:
        F.fwi_set_checkpoint(0)
    torch.cuda.synchronize()
    return [t.cpu() for t in out]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_checked_build_is_clean_and_equal(F, case):
    from paper_1804_01184_gb300 import build
    w = I.small_case(**case)
    ref = run_all(F, w)
    with F.library(build.LIB_CHECKED):
        got = run_all(F, w)            # every call checks its status: a caught access raises
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
