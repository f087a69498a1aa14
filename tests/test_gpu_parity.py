"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (from the accuracy targets of the method's FP32 path): relative L2 <= 1e-4 on
traces, <= 1e-3 on every gradient field.  The streaming kernels give each warp a strip of 120
computational columns: the small cases are narrower than one strip (95 columns at most) and
many row strips high; the multi-strip cases are 2 to 3 strips wide with a ragged last strip;
the full-size cases (681 x 681 computational cells, 6 strips) use the launch configuration
the benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_1804_01184_gb300 import inputs as I
from tests._common import GRAD_TOL, TRACE_TOL, gpu_grid, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, fwi
    build.build()
    return fwi


def run_model(F, w, a=None, b=None, **kw):
    a = w.xi_a if a is None else a
    b = w.xi_b if b is None else b
    return F.fwi_model(gpu_grid(w), w.pz, torch.from_numpy(a), torch.from_numpy(b), torch.from_numpy(w.src_xy),
                       torch.from_numpy(w.wavelet), torch.from_numpy(w.rec_xy), **kw).cpu().numpy()


CASES = [
    dict(seed=11, nx=75, nz=53, nt=300, order=8, sponge=10, ns=3, nr=9, pz=I.PZ_VP_RHO),
    dict(seed=12, nx=61, nz=70, nt=250, order=4, sponge=7, ns=2, nr=5, pz=I.PZ_IP_RHO),
    dict(seed=13, nx=40, nz=33, nt=200, order=8, sponge=0, ns=2, nr=4, pz=I.PZ_VP_IP),
    dict(seed=14, nx=66, nz=66, nt=260, order=8, sponge=12, ns=4, nr=6, pz=I.PZ_INVK_INVRHO),
    dict(seed=15, nx=50, nz=45, nt=220, order=4, sponge=5, ns=1, nr=3, pz=I.PZ_K_RHO),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_model_parity(F, case):
    w = I.small_case(**case)
    tr = run_model(F, w)
    ref = oracle.model(oracle_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    assert rel_l2(tr, ref) <= TRACE_TOL
    for s in range(w.ns):   # every shot on its own
        assert rel_l2(tr[s], ref[s]) <= TRACE_TOL


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_born_parity(F, case):
    w = I.small_case(**case)
    da = I.random_like(w.xi_a.shape, 40, 0.05)
    db = I.random_like(w.xi_a.shape, 41, 0.05)
    g = gpu_grid(w)
    dtr = F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy).cpu().numpy()
    ref = oracle.born(oracle_grid(w), w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
    assert rel_l2(dtr, ref) <= TRACE_TOL


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_gradient_parity(F, case):
    w = I.small_case(**case)
    og = oracle_grid(w)
    data = oracle.model(og, w.pz, w.xi_a * 1.4, w.xi_b * 0.6, w.src_xy, w.wavelet, w.rec_xy).astype(np.float32)
    a0, b0 = (w.xi_a * 0.5).astype(np.float32), (w.xi_b * 0.5).astype(np.float32)
    J_ref, G_ref = oracle.gradient(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
    J, G = F.fwi_gradient(gpu_grid(w), w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
    assert abs(J.item() - J_ref) <= TRACE_TOL * J_ref
    G = G.cpu().numpy()
    for pz in range(5):
        for k in range(2):
            assert rel_l2(G[pz, k], G_ref[pz, k]) <= GRAD_TOL, (pz, k, rel_l2(G[pz, k], G_ref[pz, k]))


def test_adjoint_parity_random_residual(F):
    w = I.small_case(seed=21, nx=70, nz=58, nt=240, order=8, sponge=9, ns=3, nr=8, pz=I.PZ_VP_RHO)
    res = I.random_like((w.ns, w.nr, w.nt), 5, 100.0)
    G = F.fwi_adjoint(gpu_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, res).cpu().numpy()
    G_ref = oracle.adjoint(oracle_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, res)
    for pz in range(5):
        for k in range(2):
            assert rel_l2(G[pz, k], G_ref[pz, k]) <= GRAD_TOL


@pytest.mark.parametrize("pz", range(5))
def test_dot_product_gpu(F, pz):
    """<born(dm), y> = <dm, adjoint(y)> in FP32 on the GPU."""
    w = I.small_case(seed=30 + pz, nx=64, nz=48, nt=200, order=8, sponge=8, ns=2, nr=6, pz=pz)
    g = gpu_grid(w)
    da, db = I.random_like(w.xi_a.shape, 50, 0.05), I.random_like(w.xi_a.shape, 51, 0.05)
    y = I.random_like((w.ns, w.nr, w.nt), 52, 1.0)
    Fx = F.fwi_born(g, pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy).cpu().numpy().astype(np.float64)
    G = F.fwi_adjoint(g, pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, y).cpu().numpy()
    lhs = np.sum(Fx * y)
    rhs = np.sum(G[pz, 0] * da) + np.sum(G[pz, 1] * db)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_checkpointing_and_shot_groups_match(F):
    """Plans with recomputation from checkpoints and with several shot groups give the
    gradient of the whole-history single-group plan."""
    w = I.small_case(seed=41, nx=60, nz=50, nt=300, order=8, sponge=8, ns=5, nr=6, pz=I.PZ_K_RHO)
    g = gpu_grid(w)
    data = run_model(F, w, w.xi_a * 1.3, w.xi_b * 0.8)
    a0, b0 = w.xi_a * 0.5, w.xi_b * 0.5
    full = F.workspace(g, w.ns, w.nr, F.OP_GRADIENT, 1 << 40)
    J0, G0 = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data, work=full)
    minimum = F.fwi_workspace_bytes(g, w.ns, w.nr, F.OP_GRADIENT, 0)
    for budget in (minimum, int(minimum * 1.6), int(full.numel() * 0.5)):
        work = F.workspace(g, w.ns, w.nr, F.OP_GRADIENT, budget)
        assert work.numel() <= max(budget, minimum)
        J1, G1 = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data, work=work)
        assert abs(J1.item() - J0.item()) <= 1e-12 * J0.item()
        assert rel_l2(G1.cpu().numpy(), G0.cpu().numpy()) <= 1e-6


def test_model_shot_groups_bitwise(F):
    w = I.small_case(seed=42, nx=50, nz=40, nt=150, order=8, sponge=6, ns=5, nr=4)
    g = gpu_grid(w)
    t_full = run_model(F, w)
    mn = F.fwi_workspace_bytes(g, w.ns, w.nr, F.OP_MODEL, 0)
    t_one = run_model(F, w, work=F.workspace(g, w.ns, w.nr, F.OP_MODEL, mn))
    np.testing.assert_array_equal(t_full, t_one)
    # each shot alone equals the same shot in the batch
    for s in range(w.ns):
        np.testing.assert_array_equal(run_model(F, w.subset([s]))[0], t_full[s])


# -------------------------------------------------------------------- full-size workloads

def test_config_point_full(F):
    """201 x 201 + 40-cell sponge, 4th order, 800 steps, 8 sources / 64 receivers: traces, and
    the gradient at 1400 steps (at 800 the record ends before the scattered arrivals).

    The point scatterer's residual is ~3e-4 of the traces, so the FP32 trace error (~5e-7)
    becomes a ~2e-3 error of the residual itself.  The chain forward -> residual -> adjoint is
    therefore checked link by link against the oracle: the traces at 1e-4; the adjoint given
    the oracle's residual at 1e-3; and fwi_gradient's own output against oracle.adjoint fed
    with fwi_gradient's residual (its FP32 background traces minus the data, exact in FP64),
    at 1e-3 per field, with its misfit equal to that residual's FP64 sum."""
    for nt in (800, 1400):
        w = I.config_point(nt)
        og = oracle_grid(w)
        tr = run_model(F, w)
        ref = oracle.model(og, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
        assert rel_l2(tr, ref) <= TRACE_TOL
        if nt == 800:
            continue
        a0, b0 = w.background()
        data = ref.astype(np.float32)
        bg_ref = oracle.model(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy)
        res_ref = (bg_ref - data).astype(np.float32)
        g = gpu_grid(w)
        G = F.fwi_adjoint(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, res_ref).cpu().numpy()
        G_ref = oracle.adjoint(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, res_ref)
        for pz in range(5):
            for k in range(2):
                assert rel_l2(G[pz, k], G_ref[pz, k]) <= GRAD_TOL, (pz, k)
        J, Gg = F.fwi_gradient(g, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
        Gg = Gg.cpu().numpy()
        J_ref = 0.5 * float(np.sum(res_ref.astype(np.float64) ** 2))
        assert abs(J.item() - J_ref) <= 1e-2 * J_ref            # the FP32 forward error of a tiny residual
        bg = run_model(F, w, a0, b0)                            # the traces fwi_gradient forms (bitwise)
        res64 = bg.astype(np.float64) - data.astype(np.float64)
        assert abs(J.item() - 0.5 * float(np.sum(res64 ** 2))) <= 1e-9 * J.item()
        G_own = oracle.adjoint(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, res64)
        for pz in range(5):
            for k in range(2):
                assert rel_l2(Gg[pz, k], G_own[pz, k]) <= GRAD_TOL, (pz, k, rel_l2(Gg[pz, k], G_own[pz, k]))


def test_config_gaussian_full_traces_sampled(F):
    """601 x 601, 8th order, 3000 steps, 64 sources / 256 receivers (the benchmark's launch
    configuration): all 64 shots on the GPU, shots 0 and 37 recomputed by the oracle."""
    w = I.config_gaussian(0.3, "vp")
    tr = run_model(F, w)
    assert tr.shape == (64, 256, 3000) and np.all(np.isfinite(tr))
    og = oracle_grid(w)
    for s in (0, 37):
        sub = w.subset([s])
        ref = oracle.model(og, w.pz, w.xi_a, w.xi_b, sub.src_xy, w.wavelet, w.rec_xy)[0]
        assert rel_l2(tr[s], ref) <= TRACE_TOL, s


def test_config_gaussian_full_gradient_sampled(F):
    """The benchmark's gradient at full length: 681 x 681 computational cells, 8th order, 3000
    steps, the whole-history plan; 2 of the 64 shots.  fwi_gradient at the background against
    oracle.gradient (FP64 throughout) for every field of all five parameterizations, with the
    default FP32 -> FP64 accumulation chunks.  The same gradient with one FP32 sum over the
    whole record (fwi_set_accumulation(nt)) is printed beside it for comparison."""
    w = I.config_gaussian(0.3, "vp")
    sub = w.subset([0, 37])
    og = oracle_grid(w)
    data = oracle.model(og, w.pz, w.xi_a, w.xi_b, sub.src_xy, w.wavelet, w.rec_xy).astype(np.float32)
    a0, b0 = w.background()
    J_ref, G_ref = oracle.gradient(og, w.pz, a0, b0, sub.src_xy, w.wavelet, w.rec_xy, data)
    g = gpu_grid(w)
    work = F.workspace(g, sub.ns, w.nr, F.OP_GRADIENT)
    assert work.numel() >= F.fwi_workspace_bytes(g, sub.ns, w.nr, F.OP_GRADIENT, 1 << 45)   # whole history
    err = {}
    try:
        for acc in (0, w.nt):
            F.fwi_set_accumulation(acc)
            J, G = F.fwi_gradient(g, w.pz, a0, b0, sub.src_xy, w.wavelet, w.rec_xy, data, work=work)
            G = G.cpu().numpy()
            err[acc] = (abs(J.item() - J_ref) / J_ref,
                        [[rel_l2(G[pz, k], G_ref[pz, k]) for k in range(2)] for pz in range(5)])
    finally:
        F.fwi_set_accumulation(0)
    for acc, (ej, eg) in err.items():
        print(f"accumulation {'64-step chunks' if acc == 0 else 'one FP32 sum'}: misfit rel err {ej:.2e}, "
              f"gradient rel L2 max {np.max(eg):.2e} per field {np.round(np.array(eg), 7).tolist()}")
    ej, eg = err[0]
    assert ej <= TRACE_TOL
    assert np.max(eg) <= GRAD_TOL


def test_accumulation_chunks_agree(F):
    """Every accumulation chunk length gives the same gradient to FP32 rounding (the chunk only
    decides when FP32 partial sums move into FP64), each within the tolerance of the oracle,
    and a given length is bitwise reproducible."""
    w = I.small_case(seed=25, nx=60, nz=52, nt=230, order=8, sponge=8, ns=3, nr=7, pz=I.PZ_IP_RHO)
    g = gpu_grid(w)
    data = I.random_like((w.ns, w.nr, w.nt), 26, 1e3)
    ref = oracle.gradient(oracle_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)[1]
    out = {}
    try:
        for acc in (1, 7, 64, 229, 230, 10000):
            F.fwi_set_accumulation(acc)
            out[acc] = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)[1].cpu().numpy()
        F.fwi_set_accumulation(7)
        again = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)[1].cpu().numpy()
        np.testing.assert_array_equal(again, out[7])
        with pytest.raises(F.FwiError):
            F.fwi_set_accumulation(-1)
    finally:
        F.fwi_set_accumulation(0)
    for acc, G in out.items():
        assert rel_l2(G, out[64]) <= 1e-5, acc
        for pz in range(5):
            for k in range(2):
                assert rel_l2(G[pz, k], ref[pz, k]) <= GRAD_TOL, (acc, pz, k)


@pytest.mark.parametrize("order", [4, 8])
def test_born_multi_strip(F, order):
    """Born modelling on grids 2 and 3 warp strips wide (the last strip ragged), through
    fwi_born and through the batching engine, against the oracle."""
    from paper_1804_01184_gb300 import engine as E
    cases = [dict(seed=70 + order, nx=150, nz=47, nt=210, order=order, sponge=9, ns=2, nr=6, pz=I.PZ_VP_RHO),
             dict(seed=80 + order, nx=231, nz=38, nt=160, order=order, sponge=5, ns=3, nr=5, pz=I.PZ_K_RHO)]
    eng = E.Engine(1 << 30)
    try:
        for case in cases:
            w = I.small_case(**case)
            assert w.Nx > 120 * (1 if case["nx"] < 200 else 2)
            g = gpu_grid(w)
            da = I.random_like(w.xi_a.shape, case["seed"] + 1, 0.05)
            db = I.random_like(w.xi_a.shape, case["seed"] + 2, 0.05)
            ref = oracle.born(oracle_grid(w), w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
            dtr = F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
            assert rel_l2(dtr.cpu().numpy(), ref) <= TRACE_TOL
            for s in range(w.ns):
                assert rel_l2(dtr[s].cpu().numpy(), ref[s]) <= TRACE_TOL
            with torch.cuda.stream(eng.stream):
                t = eng.submit_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy)
            res = {r.ticket: r for r in eng.drain()}
            torch.cuda.synchronize()
            assert torch.equal(res[t].traces, dtr)
    finally:
        eng.close()


def test_config_gaussian_full_adjoint_sampled(F):
    """Full 681 x 681 computational grid and 8th order; a random residual on 2 shots over 400
    steps (the oracle keeps the whole FP64 history in host memory)."""
    w = I.config_gaussian(0.3, "rho", nt=400)
    sub = w.subset([5, 50])
    res = I.random_like((2, w.nr, w.nt), 77, 1e3)
    G = F.fwi_adjoint(gpu_grid(w), w.pz, w.xi_a, w.xi_b, sub.src_xy, w.wavelet, w.rec_xy, res).cpu().numpy()
    G_ref = oracle.adjoint(oracle_grid(w), w.pz, w.xi_a, w.xi_b, sub.src_xy, w.wavelet, w.rec_xy, res)
    for pz in range(5):
        for k in range(2):
            assert rel_l2(G[pz, k], G_ref[pz, k]) <= GRAD_TOL


# ---------------------------------------------------------------------------- edge cases

def test_empty_shots_and_receivers(F):
    w = I.small_case(seed=50, nx=30, nz=30, nt=50, ns=2, nr=3)
    g = gpu_grid(w)
    none_s = np.zeros((0, 2), np.float32)
    tr = F.fwi_model(g, w.pz, w.xi_a, w.xi_b, none_s, w.wavelet, w.rec_xy)
    assert tr.shape == (0, w.nr, w.nt)
    tr = F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, none_s)
    assert tr.shape == (w.ns, 0, w.nt)
    J, G = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, none_s, w.wavelet, w.rec_xy, np.zeros((0, w.nr, w.nt), np.float32))
    assert J.item() == 0.0 and torch.all(G == 0)
    J, G = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, none_s, np.zeros((w.ns, 0, w.nt), np.float32))
    assert J.item() == 0.0 and torch.all(G == 0)


def test_zero_residual_gives_zero_gradient(F):
    w = I.small_case(seed=51, nx=40, nz=40, nt=120, ns=2, nr=5)
    data = run_model(F, w)
    J, G = F.fwi_gradient(gpu_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)
    assert J.item() == 0.0 and torch.all(G == 0)


def test_errors_reported(F):
    w = I.small_case(seed=52, nx=30, nz=30, nt=40, ns=1, nr=2)
    g = gpu_grid(w)
    bad = w.xi_a.copy()
    bad[3, 4] = -1.5
    with pytest.raises(F.FwiError) as e:
        F.fwi_model(g, w.pz, bad, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    assert e.value.code == -1
    with pytest.raises(F.FwiError) as e:     # dt far above the stability limit
        F.fwi_model(gpu_grid(w, dt=5e-3), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet[:40], w.rec_xy)
    assert e.value.code == -2
    with pytest.raises(F.FwiError) as e:     # receiver outside the physical grid
        F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, np.array([[1e4, 0.0]], np.float32))
    assert e.value.code == -1
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FwiError) as e:
        F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, work=small)
    assert e.value.code == -3
    # the context is still usable
    run_model(F, w)


@pytest.mark.parametrize("order", [4, 8])
def test_poisoned_workspace_gives_identical_results(F, order):
    """A workspace full of NaN bytes before every call gives bit-identical traces, Born traces
    and gradients: no kernel reads memory that the operation has not written."""
    w = I.small_case(seed=60 + order, nx=37, nz=29, nt=90, order=order, sponge=5, ns=3, nr=4)
    g = gpu_grid(w)
    da, db = I.random_like(w.xi_a.shape, 1, 0.05), I.random_like(w.xi_a.shape, 2, 0.05)
    data = run_model(F, w, w.xi_a * 1.2, w.xi_b * 0.9)
    out = []
    for poison in (False, True):
        ws = {op: F.workspace(g, w.ns, w.nr, op, 1 << 34) for op in (F.OP_MODEL, F.OP_BORN, F.OP_GRADIENT)}
        if poison:
            for t in ws.values():
                t.fill_(0xFF)       # every float32 becomes NaN
        tr = run_model(F, w, work=ws[F.OP_MODEL])
        bo = F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy,
                        work=ws[F.OP_BORN]).cpu().numpy()
        J, G = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data, work=ws[F.OP_GRADIENT])
        out.append((tr, bo, J.item(), G.cpu().numpy()))
    (t0, b0, J0, G0), (t1, b1, J1, G1) = out
    assert np.all(np.isfinite(t1)) and np.all(np.isfinite(b1)) and np.all(np.isfinite(G1))
    np.testing.assert_array_equal(t0, t1)
    np.testing.assert_array_equal(b0, b1)
    assert J0 == J1
    np.testing.assert_array_equal(G0, G1)


def test_adjoint_with_receivers_sharing_cells_is_deterministic(F):
    """Receivers on the same or neighbouring nodes share footprint cells: the adjoint source
    of a cell is summed in receiver order (no atomics), so repeated runs agree bitwise, and
    the result still matches the oracle."""
    w = I.small_case(seed=21, nx=48, nz=40, nt=160, order=8, sponge=6, ns=2, nr=4)
    base = w.rec_xy[:2]
    rec = np.concatenate([base, base, base + np.float32(1.0), base + np.float32([2.5, 0.0]),
                          base + np.float32([5.0, 5.0])]).astype(np.float32)   # 10 receivers
    w.rec_xy = rec
    res = I.random_like((w.ns, w.nr, w.nt), 22, 1.0)
    g = gpu_grid(w)
    runs = [F.fwi_adjoint(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, res).cpu() for _ in range(3)]
    assert torch.equal(runs[0], runs[1]) and torch.equal(runs[0], runs[2])
    ref = oracle.adjoint(oracle_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, res)
    G = runs[0].numpy()
    for pz in range(5):
        for k in range(2):
            assert rel_l2(G[pz, k], ref[pz, k]) <= GRAD_TOL


def test_strip_heights_give_bitwise_identical_results(F):
    """The strip height only partitions the grid among warps: every height (fixed, or chosen
    per launch) gives bitwise identical traces, Born traces and gradients."""
    w = I.small_case(seed=23, nx=70, nz=83, nt=120, order=8, sponge=6, ns=3, nr=5)
    g = gpu_grid(w)
    da, db = I.random_like(w.xi_a.shape, 3, 0.05), I.random_like(w.xi_a.shape, 4, 0.05)
    data = I.random_like((w.ns, w.nr, w.nt), 5, 1e3)
    out = []
    try:
        for tz in (0, 8, 13, 16, 24, 36, 64, 200):
            F.fwi_set_tile(tz, 0)
            tr = run_model(F, w)
            bo = F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy).cpu().numpy()
            J, G = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)
            out.append((tr, bo, J.item(), G.cpu().numpy()))
    finally:
        F.fwi_set_tile(0, 0)
    for o in out[1:]:
        np.testing.assert_array_equal(o[0], out[0][0])
        np.testing.assert_array_equal(o[1], out[0][1])
        assert o[2] == out[0][2]
        np.testing.assert_array_equal(o[3], out[0][3])


@pytest.mark.parametrize("variant", [1, 2])
def test_register_capped_variants_are_bitwise_identical(F, variant):
    """The register-capped builds of the streaming kernels (fwi_set_tile's variant) compute
    the same arithmetic: traces, Born traces and gradients equal the default build bitwise."""
    w = I.small_case(seed=24, nx=64, nz=58, nt=110, order=8, sponge=6, ns=2, nr=5)
    g = gpu_grid(w)
    da, db = I.random_like(w.xi_a.shape, 6, 0.05), I.random_like(w.xi_a.shape, 7, 0.05)
    data = I.random_like((w.ns, w.nr, w.nt), 8, 1e3)
    out = []
    try:
        for v in (0, variant):
            F.fwi_set_tile(0, v)
            tr = run_model(F, w)
            bo = F.fwi_born(g, w.pz, w.xi_a, w.xi_b, da, db, w.src_xy, w.wavelet, w.rec_xy).cpu().numpy()
            J, G = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data)
            out.append((tr, bo, J.item(), G.cpu().numpy()))
    finally:
        F.fwi_set_tile(0, 0)
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])
    assert out[1][2] == out[0][2]
    np.testing.assert_array_equal(out[1][3], out[0][3])


def test_profile_sampling_counts_every_launch_and_times_one_in_n(F):
    """fwi_profile(N) times the first of every N launches of each kernel and still counts them
    all: the report's launches equal the library's launch count, the timed ones ceil(n / N)."""
    import ctypes
    w = I.small_case(seed=2, nx=40, nz=36, nt=37, order=8, sponge=6, ns=2, nr=5)
    g = gpu_grid(w)
    F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)     # plans, tuner state
    torch.cuda.synchronize()
    L = F.lib()
    L.fwi_profile(4)
    F.launch_count()
    F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    launched = F.launch_count()
    torch.cuda.synchronize()
    L.fwi_profile(0)
    buf = ctypes.create_string_buffer(1 << 16)
    assert L.fwi_profile_report(buf, len(buf)) > 0
    total = 0
    for line in buf.value.decode().splitlines():
        name, seen, timed, ms = line.rsplit(" ", 3)
        seen, timed = int(seen), int(timed)
        assert timed == (seen + 3) // 4, line
        assert float(ms) > 0
        total += seen
    assert total == launched


def test_trace_ranges_per_phase(F):
    """fwi_trace(1): one NVTX range per phase -- the model build, each group's forward, each
    checkpoint segment's recompute and adjoint, the reduction; results unchanged."""
    w = I.small_case(seed=27, nx=44, nz=40, nt=90, order=8, sponge=5, ns=3, nr=4)
    g = gpu_grid(w)
    data = I.random_like((w.ns, w.nr, w.nt), 28, 1e3)
    try:
        F.fwi_set_checkpoint(30)                      # 3 segments
        work = F.workspace(g, 2, w.nr, F.OP_GRADIENT, 1 << 40)   # sized for 2 shots: several groups
        G0 = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data, work=work)[1].clone()
        F.trace_report()
        F.fwi_trace(True)
        G1 = F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, data, work=work)[1]
        F.fwi_born(g, w.pz, w.xi_a, w.xi_b, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
        rep = F.trace_report()
    finally:
        F.fwi_trace(False)
        F.fwi_set_checkpoint(0)
    assert torch.equal(G0, G1)
    groups = rep["fwi:forward"]                       # one forward range per shot group
    assert groups >= 2
    assert rep["fwi:model_build"] == 2                # the gradient and the Born call
    assert rep["fwi:adjoint"] == groups * 3
    assert rep["fwi:recompute"] == groups * 2
    assert rep["fwi:reduce"] == 1
    assert rep["fwi:born"] >= 1
