"""Batching engine (fwi_engine_* in the C ABI): many independent jobs of different grids,
stencil orders, shot counts, lengths and kinds run together, one batched launch per wave
family and time step.  Every job's result must be bitwise equal to the single-job call with
the same plan -- alone in the engine and in a mix -- and the engine must admit work as the
arena frees, split batches wider than one launch's table, and refuse invalid jobs."""
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
    from paper_1804_01184_gb300 import build, engine, fwi
    build.build()
    return fwi, engine


# uneven jobs: (kind, small_case kwargs, work_budget)
MIX = [
    ("model", dict(seed=101, nx=75, nz=53, nt=180, order=8, sponge=10, ns=3, nr=9, pz=I.PZ_VP_RHO), 0),
    ("model", dict(seed=102, nx=40, nz=61, nt=95, order=4, sponge=6, ns=1, nr=4, pz=I.PZ_K_RHO), 1 << 30),
    ("born", dict(seed=103, nx=66, nz=48, nt=150, order=8, sponge=8, ns=2, nr=5, pz=I.PZ_IP_RHO), 0),
    ("born", dict(seed=104, nx=51, nz=51, nt=120, order=4, sponge=5, ns=3, nr=3, pz=I.PZ_VP_IP), 1 << 30),
    ("gradient", dict(seed=105, nx=58, nz=50, nt=200, order=8, sponge=8, ns=3, nr=7, pz=I.PZ_VP_RHO), 0),
    ("gradient", dict(seed=106, nx=45, nz=37, nt=140, order=4, sponge=6, ns=2, nr=6, pz=I.PZ_INVK_INVRHO), 1 << 30),
    ("gradient", dict(seed=107, nx=70, nz=44, nt=230, order=8, sponge=0, ns=4, nr=5, pz=I.PZ_K_RHO), 0),
    ("model", dict(seed=108, nx=33, nz=90, nt=60, order=8, sponge=4, ns=5, nr=2, pz=I.PZ_INVK_INVRHO), 0),
]

OPS = {"model": 0, "born": 1, "gradient": 3}


def make_inputs(kind, case):
    w = I.small_case(**case)
    extra = {}
    if kind == "born":
        extra["dxi"] = (I.random_like(w.xi_a.shape, case["seed"] + 1000, 0.05),
                        I.random_like(w.xi_a.shape, case["seed"] + 2000, 0.05))
    if kind == "gradient":
        extra["data"] = I.random_like((w.ns, w.nr, w.nt), case["seed"] + 3000, 1e-3)
    return w, extra


def single(F, kind, w, extra, budget):
    g = gpu_grid(w)
    nbytes = F.fwi_workspace_bytes(g, w.ns, w.nr, OPS[kind], budget)
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    if kind == "model":
        return (F.fwi_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, work=work),)
    if kind == "born":
        return (F.fwi_born(g, w.pz, w.xi_a, w.xi_b, *extra["dxi"], w.src_xy, w.wavelet, w.rec_xy, work=work),)
    return F.fwi_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, extra["data"], work=work)


def submit(E, kind, w, extra, budget):
    g = gpu_grid(w)
    if kind == "model":
        return E.submit_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, work_budget=budget)
    if kind == "born":
        return E.submit_born(g, w.pz, w.xi_a, w.xi_b, *extra["dxi"], w.src_xy, w.wavelet, w.rec_xy,
                             work_budget=budget)
    return E.submit_gradient(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy, extra["data"],
                             work_budget=budget)


def outputs(r):
    return (r.traces,) if r.traces is not None else (r.misfit, r.grads)


def assert_same(a, b):
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert x.shape == y.shape and x.dtype == y.dtype
        assert torch.equal(x, y), (x.double() - y.double()).abs().max().item()


def test_mix_matches_single_calls_and_jobs_alone(L):
    F, Eng = L
    jobs = [(k, *make_inputs(k, c), b) for k, c, b in MIX]
    refs = [single(F, k, w, x, b) for k, w, x, b in jobs]
    # the whole mix in one engine, its arena full of NaN bytes: no job reads what it has not written
    E = Eng.Engine(4 << 30)
    E.arena.fill_(0xFF)
    torch.cuda.synchronize()
    tickets = [submit(E, k, w, x, b) for k, w, x, b in jobs]
    res = {r.ticket: r for r in E.drain(64)}
    assert sorted(res) == sorted(tickets)
    assert E.info() == dict(queued=0, running=0, pending=0, arena_used=0)
    for t, ref in zip(tickets, refs):
        assert_same(outputs(res[t]), ref)
    # each job alone
    for (k, w, x, b), ref in zip(jobs[::3], refs[::3]):
        E1 = Eng.Engine(1 << 30)
        t = submit(E1, k, w, x, b)
        (r,) = E1.drain()
        assert r.ticket == t
        assert_same(outputs(r), ref)
        E1.close()
    E.close()


def test_engine_gradient_against_oracle(L):
    F, Eng = L
    k, case, b = MIX[4]
    w = I.small_case(**case)
    og = oracle_grid(w)
    data = oracle.model(og, w.pz, w.xi_a * 1.4, w.xi_b * 0.6, w.src_xy, w.wavelet, w.rec_xy).astype(np.float32)
    a0, b0 = (w.xi_a * 0.5).astype(np.float32), (w.xi_b * 0.5).astype(np.float32)
    E = Eng.Engine(1 << 30)
    E.submit_model(gpu_grid(w), w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)      # a neighbour
    t = E.submit_gradient(gpu_grid(w), w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
    r = {x.ticket: x for x in E.drain()}[t]
    J_ref, G_ref = oracle.gradient(og, w.pz, a0, b0, w.src_xy, w.wavelet, w.rec_xy, data)
    assert abs(r.misfit.item() - J_ref) <= TRACE_TOL * J_ref
    G = r.grads.cpu().numpy()
    for pz in range(5):
        for c in range(2):
            assert rel_l2(G[pz, c], G_ref[pz, c]) <= GRAD_TOL


def test_admission_under_arena_pressure(L):
    F, Eng = L
    kind, case, _ = MIX[4]
    variants = [dict(case, seed=200 + s) for s in range(6)]
    jobs = [(kind, *make_inputs(kind, c), 0) for c in variants]
    need = F.fwi_workspace_bytes(gpu_grid(jobs[0][1]), jobs[0][1].ns, jobs[0][1].nr, OPS[kind], 0)
    E = Eng.Engine(2 * need + need // 2)           # room for two jobs at a time
    E.arena.fill_(0xFF)
    torch.cuda.synchronize()
    tickets = [submit(E, k, w, x, b) for k, w, x, b in jobs]
    E.run(1)
    st = E.info()
    assert st["running"] == 2 and st["queued"] == 4 and st["arena_used"] <= 2 * need + need // 2
    res = {r.ticket: r for r in E.drain(32)}
    assert sorted(res) == tickets
    assert E.info()["arena_used"] == 0
    for t, (k, w, x, b) in zip(tickets, jobs):
        assert_same(outputs(res[t]), single(F, k, w, x, b))
    E.close()


def test_more_jobs_than_one_launch_table(L):
    F, Eng = L
    E = Eng.Engine(2 << 30)
    jobs = []
    for s in range(130):                                 # > 96 jobs per wave family
        case = dict(seed=300 + s, nx=24 + s % 7, nz=20 + s % 5, nt=30 + s % 11, order=4 if s % 10 == 0 else 8, sponge=3,
                    ns=1 + s % 3, nr=2, pz=s % 5)
        jobs.append(("model", *make_inputs("model", case), 0))
    tickets = [submit(E, k, w, x, b) for k, w, x, b in jobs]
    E.run(1)
    assert E.info()["running"] == 130
    res = {r.ticket: r for r in E.drain()}
    for t, (k, w, x, b) in zip(tickets, jobs):
        assert_same(outputs(res[t]), single(F, k, w, x, b))
    E.close()


def test_invalid_jobs_are_refused(L):
    F, Eng = L
    w = I.small_case(seed=400)
    g = gpu_grid(w)
    E = Eng.Engine(64 << 20)
    with pytest.raises(F.FwiError) as e:             # CFL-free but unknown parameterization
        E.submit_model(g, 7, w.xi_a, w.xi_b, w.src_xy, w.wavelet, w.rec_xy)
    assert e.value.code == -1
    big = F.make_grid(2001, 2001, 2.5, 2.5e-4, 100, order=8, sponge=40)
    z = torch.zeros((2001, 2001), device="cuda")
    xy = torch.tensor([[2500.0, 2500.0]], device="cuda")
    with pytest.raises(F.FwiError) as e:             # workspace larger than the arena
        E.submit_model(big, 0, z, z, xy, torch.zeros(100, device="cuda"), xy)
    assert e.value.code == -3
    assert E.info() == dict(queued=0, running=0, pending=0, arena_used=0)
    E.close()


def test_degenerate_jobs_and_a_job_filling_the_arena(L):
    """Jobs without receivers or without shots finish with the single calls' results; a job
    whose workspace is the whole arena waits until the jobs ahead of it retire, then runs."""
    F, Eng = L
    w = I.small_case(seed=500, nx=40, nz=36, nt=70, order=8, sponge=4, ns=2, nr=3)
    g = gpu_grid(w)
    none = np.zeros((0, 2), np.float32)
    big = I.small_case(seed=501, nx=90, nz=80, nt=90, order=4, sponge=6, ns=3, nr=4)
    data = I.random_like((big.ns, big.nr, big.nt), 502, 1e-3)
    need = F.fwi_workspace_bytes(gpu_grid(big), big.ns, big.nr, F.OP_GRADIENT, 0)
    E = Eng.Engine(need)
    t_norec = E.submit_model(g, w.pz, w.xi_a, w.xi_b, w.src_xy, w.wavelet, none)
    t_nosrc = E.submit_gradient(g, w.pz, w.xi_a, w.xi_b, none, w.wavelet, w.rec_xy,
                                np.zeros((0, w.nr, w.nt), np.float32))
    t_big = E.submit_gradient(gpu_grid(big), big.pz, big.xi_a, big.xi_b, big.src_xy, big.wavelet, big.rec_xy, data)
    E.run(1)
    assert E.info()["queued"] >= 1                     # the big job waits for the arena
    res = {r.ticket: r for r in E.drain()}
    assert res[t_norec].traces.shape == (w.ns, 0, w.nt)
    torch.cuda.synchronize()
    assert res[t_nosrc].misfit.item() == 0.0 and not torch.any(res[t_nosrc].grads != 0)
    assert_same(outputs(res[t_big]), single(F, "gradient", big, {"data": data}, 0))
    E.close()


def test_many_gradients_overflow_the_per_receiver_table(L):
    """More adjoint jobs than one forward launch's per-receiver table holds (40): the rest of
    the injections go out in their own launches; every result equals the single call."""
    F, Eng = L
    E = Eng.Engine(2 << 30)
    jobs = []
    for s in range(56):
        case = dict(seed=600 + s, nx=26 + s % 5, nz=22 + s % 3, nt=24 + s % 7, order=8, sponge=3, ns=1 + s % 2,
                    nr=3, pz=s % 5)
        jobs.append(("gradient", *make_inputs("gradient", case), 0))
    jobs.append(("model", *make_inputs("model", dict(seed=700, nx=30, nz=30, nt=60, ns=2, nr=3)), 0))
    tickets = [submit(E, k, w, x, b) for k, w, x, b in jobs]
    res = {r.ticket: r for r in E.drain()}
    for t, (k, w, x, b) in zip(tickets, jobs):
        assert_same(outputs(res[t]), single(F, k, w, x, b))
    E.close()


def test_cancel_running_and_queued_jobs(L):
    """fwi_engine_cancel: a running job stops, its arena block is free at once and its ticket
    never comes back; a queued job leaves the queue; every other job's result equals the single
    call bitwise, also the job admitted into the cancelled job's memory."""
    F, Eng = L
    kind, case, _ = MIX[4]
    jobs = [(kind, *make_inputs(kind, dict(case, seed=800 + s)), 0) for s in range(5)]
    need = F.fwi_workspace_bytes(gpu_grid(jobs[0][1]), jobs[0][1].ns, jobs[0][1].nr, OPS[kind], 0)
    E = Eng.Engine(2 * need + need // 2)           # room for two jobs at a time
    E.arena.fill_(0xFF)
    torch.cuda.synchronize()
    tickets = [submit(E, k, w, x, b) for k, w, x, b in jobs]
    E.run(3)                                        # jobs 0 and 1 are running, 2..4 queued
    st = E.info()
    assert st["running"] == 2 and st["queued"] == 3
    used = st["arena_used"]
    E.cancel(tickets[1])                            # running
    assert E.info()["running"] == 1 and E.info()["arena_used"] < used
    E.cancel(tickets[3])                            # queued (admission waits for the next run)
    assert E.info()["queued"] == 2
    with pytest.raises(F.FwiError):
        E.cancel(tickets[1])                        # already cancelled
    res = {r.ticket: r for r in E.drain(16)}
    assert sorted(res) == [tickets[0], tickets[2], tickets[4]]
    assert E.info()["arena_used"] == 0
    for t in (0, 2, 4):
        k, w, x, b = jobs[t]
        assert_same(outputs(res[tickets[t]]), single(F, k, w, x, b))
    with pytest.raises(F.FwiError):
        E.cancel(tickets[0])                        # finished
    E.close()
