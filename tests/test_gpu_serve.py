"""Continuous batching: a seeded Poisson stream of forward, Born and gradient requests on
different grids, served through the engine while earlier requests are still on the GPU.
Every result must equal (bitwise) the single-job call with the same plan -- the result the
request gets alone -- and the smallest requests must match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests._common import GRAD_TOL, TRACE_TOL, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = dict(side=(40, 90), steps=(80, 200), shots=(1, 3))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_01184_gb300 import build, engine, fwi, serve, workloads
    build.build()
    return fwi, engine, serve, workloads


ARENA = 2 << 30


def single(F, Eng, S, r):
    w = r.workload
    g = F.make_grid(**w.grid_kwargs())
    op = {Eng.JOB_MODEL: F.OP_MODEL, Eng.JOB_BORN: F.OP_BORN, Eng.JOB_GRADIENT: F.OP_GRADIENT}[r.kind]
    budget = S.default_budget(ARENA) if r.work_budget is None else r.work_budget
    work = torch.empty(F.fwi_workspace_bytes(g, w.ns, w.nr, op, budget), dtype=torch.uint8, device="cuda")
    if r.kind == Eng.JOB_MODEL:
        return (F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, work=work),)
    if r.kind == Eng.JOB_BORN:
        return (F.fwi_born(g, w.pz, w.xi_a, w.xi_b, *r.dxi, w.src_xy, w.wavelet, w.rec_xy, work=work),)
    return F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, r.data, work=work)


def test_stream_results_equal_alone_and_oracle(L):
    F, Eng, S, W = L
    from paper_1804_01184_gb300 import inputs as I
    reqs = W.serve_requests(18, seed=9, **SIZES)
    for r in reqs[::4]:
        r.work_budget = 0                                  # some requests on their smallest plan
    arrivals = I.poisson_arrivals(len(reqs), 400.0, seed=3)
    stats, results = S.serve(reqs, arrivals, ARENA, keep_results=True)
    assert stats["requests"] == len(reqs) and all(r is not None for r in results)
    assert stats["max_running"] >= 2                      # requests overlapped on the GPU
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    torch.cuda.synchronize()
    for r, res in zip(reqs, results):
        ref = single(F, Eng, S, r)
        got = (res.traces,) if res.traces is not None else (res.misfit, res.grads)
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
    # the smallest request of each kind against the FP64 oracle
    for kind in (Eng.JOB_MODEL, Eng.JOB_BORN, Eng.JOB_GRADIENT):
        ks = [k for k, r in enumerate(reqs) if r.kind == kind]
        if not ks:
            continue
        k = min(ks, key=lambda k: W.cells(reqs[k].workload))
        r, res, w = reqs[k], results[k], reqs[k].workload
        g = oracle.make_grid(**w.grid_kwargs())
        if kind == Eng.JOB_MODEL:
            ref = oracle.model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
            assert rel_l2(res.traces.cpu().numpy(), ref) <= TRACE_TOL
        elif kind == Eng.JOB_BORN:
            ref = oracle.born(g, w.pz, w.xi_a, w.xi_b, *r.dxi, w.src_xy, w.wavelet, w.rec_xy)
            assert rel_l2(res.traces.cpu().numpy(), ref) <= TRACE_TOL
        else:
            J, G = oracle.gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, r.data)
            assert abs(res.misfit.item() - J) <= TRACE_TOL * J
            got = res.grads.cpu().numpy()
            for pz in range(5):
                for c in range(2):
                    assert rel_l2(got[pz, c], G[pz, c]) <= GRAD_TOL


def test_deadlines_cancel_requests_and_leave_the_rest_unchanged(L):
    """Requests whose deadline passes are cancelled in the engine (queued or running); the
    others finish with the results they get alone."""
    F, Eng, S, W = L
    from paper_1804_01184_gb300 import inputs as I
    reqs = W.serve_requests(12, seed=19, **SIZES)
    for r in reqs[1::3]:
        r.deadline_s = 0.0                                 # cancelled on the loop's next pass
    arrivals = I.poisson_arrivals(len(reqs), 400.0, seed=4)
    stats, results = S.serve(reqs, arrivals, ARENA, keep_results=True)
    gone = [k for k in range(len(reqs)) if results[k] is None]
    assert stats["cancelled"] == len(gone) >= 1
    assert set(gone) <= set(range(1, len(reqs), 3))
    torch.cuda.synchronize()
    for r, res in zip(reqs, results):
        if res is None:
            continue
        ref = single(F, Eng, S, r)
        got = (res.traces,) if res.traces is not None else (res.misfit, res.grads)
        for x, y in zip(got, ref):
            assert torch.equal(x, y)
