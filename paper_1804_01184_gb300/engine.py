"""Python binding of the batching engine of libfwi.so (``fwi_engine_*`` in include/fwi.h).

Argument marshalling only.  An :class:`Engine` owns a device arena (a torch uint8 tensor)
and a stream; jobs (forward modelling, Born modelling, misfit + gradient) are submitted
with the same arguments as the single-job calls in :mod:`.fwi`, run together -- one batched
launch per wave family and time step -- and come back by ticket.  The engine keeps every
tensor a job uses alive until the job is reported done.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import torch

from . import fwi as F

JOB_MODEL, JOB_BORN, JOB_GRADIENT = range(3)


class _Job(C.Structure):
    """Mirror of ``fwi_job``."""

    _fields_ = [
        ("kind", C.c_int), ("grid", F.Grid), ("pz", C.c_int),
        ("xi_a", C.c_void_p), ("xi_b", C.c_void_p), ("dxi_a", C.c_void_p), ("dxi_b", C.c_void_p),
        ("src", F._Sources), ("rec", F._Receivers),
        ("traces", C.c_void_p), ("data", C.c_void_p), ("misfit", C.c_void_p), ("grads", C.c_void_p),
        ("work_budget", C.c_size_t),
    ]


_bound = False


def _lib():
    global _bound
    L = F.lib()
    if not _bound:
        vp = C.c_void_p
        L.fwi_engine_create.argtypes = [C.POINTER(vp), vp, C.c_size_t, vp]
        L.fwi_engine_submit.argtypes = [vp, C.POINTER(_Job), C.POINTER(C.c_longlong)]
        L.fwi_engine_run.argtypes = [vp, C.c_int, C.POINTER(C.c_longlong), C.c_int, C.POINTER(C.c_int)]
        L.fwi_engine_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_size_t)]
        L.fwi_engine_destroy.argtypes = [vp]
        L.fwi_engine_cancel.argtypes = [vp, C.c_longlong]
        _bound = True
    return L


@dataclasses.dataclass
class Result:
    """Outputs of a finished job: traces (MODEL, BORN) or misfit + grads (GRADIENT)."""
    ticket: int
    kind: int
    traces: torch.Tensor | None = None
    misfit: torch.Tensor | None = None
    grads: torch.Tensor | None = None


class Engine:
    """Many independent jobs in one arena (see fwi_engine_* in include/fwi.h)."""

    def __init__(self, arena_bytes: int, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        self._h = C.c_void_p()
        F._raise(_lib().fwi_engine_create(C.byref(self._h), C.c_void_p(self.arena.data_ptr()),
                                          self.arena.numel(), C.c_void_p(self.stream.cuda_stream)))
        self._jobs: dict[int, tuple] = {}
        self._cancelled: list[tuple] = []   # (event, tensors) of cancelled jobs still on the stream

    # ---------------------------------------------------------------- submission
    def _submit(self, kind, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, dxi=None, out=None, data=None,
                work_budget=0):
        with torch.cuda.stream(self.stream):
            a, b = F._dev(xi_a), F._dev(xi_b)
            keep, S, R = F._acq(src_xy, wavelet, rec_xy)
            J = _Job()
            J.kind, J.grid, J.pz, J.work_budget = kind, grid, int(pz), int(work_budget)
            J.xi_a, J.xi_b, J.src, J.rec = a.data_ptr(), b.data_ptr(), S, R
            res = Result(0, kind)
            held = [a, b, keep]
            if kind == JOB_BORN:
                da, db = F._dev(dxi[0]), F._dev(dxi[1])
                J.dxi_a, J.dxi_b = da.data_ptr(), db.data_ptr()
                held += [da, db]
            if kind in (JOB_MODEL, JOB_BORN):
                res.traces = out if out is not None else torch.empty((S.ns, R.nr, grid.nt), dtype=torch.float32,
                                                                     device="cuda")
                J.traces = res.traces.data_ptr()
            else:
                d = F._dev(data)
                res.misfit = torch.empty((), dtype=torch.float64, device="cuda")
                res.grads = torch.empty((5, 2, grid.nz, grid.nx), dtype=torch.float64, device="cuda")
                J.data, J.misfit, J.grads = d.data_ptr(), res.misfit.data_ptr(), res.grads.data_ptr()
                held.append(d)
        # inputs made on the engine's stream are ordered before the job's kernels
        t = C.c_longlong()
        F._raise(_lib().fwi_engine_submit(self._h, C.byref(J), C.byref(t)))
        res.ticket = int(t.value)
        self._jobs[res.ticket] = (res, held)
        return res.ticket

    # work_budget: the job runs the plan fwi_workspace_bytes(grid, ns, nr, op, work_budget)
    # gives (0: the smallest plan) -- bitwise what the single-job call computes with that
    # workspace.
    def submit_model(self, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, traces=None, work_budget=0) -> int:
        return self._submit(JOB_MODEL, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, out=traces,
                            work_budget=work_budget)

    def submit_born(self, grid, pz, xi_a, xi_b, dxi_a, dxi_b, src_xy, wavelet, rec_xy, dtraces=None,
                    work_budget=0) -> int:
        return self._submit(JOB_BORN, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, dxi=(dxi_a, dxi_b), out=dtraces,
                            work_budget=work_budget)

    def submit_gradient(self, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, data, work_budget=0) -> int:
        return self._submit(JOB_GRADIENT, grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, data=data,
                            work_budget=work_budget)

    def cancel(self, ticket: int):
        """Cancels a queued or running job (fwi_engine_cancel): it never comes back from run();
        its tensors are kept until the engine's stream has passed the cancellation."""
        F._raise(_lib().fwi_engine_cancel(self._h, int(ticket)))
        res, held = self._jobs.pop(int(ticket))
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self._cancelled.append((ev, (res, held)))

    # ------------------------------------------------------------------- running
    def run(self, iterations: int = 64, max_done: int = 4096) -> list[Result]:
        """Advances the engine; returns the jobs that finished (results complete on the device,
        ordered before later work on the engine's stream)."""
        self._cancelled = [c for c in self._cancelled if not c[0].query()]
        done = (C.c_longlong * max_done)()
        nd = C.c_int()
        F._raise(_lib().fwi_engine_run(self._h, int(iterations), done, int(max_done), C.byref(nd)))
        out = []
        for k in range(nd.value):
            res, _ = self._jobs.pop(int(done[k]))
            out.append(res)
        return out

    def drain(self, iterations: int = 256) -> list[Result]:
        """Runs until every submitted job has finished."""
        out = []
        while self._jobs:
            out += self.run(iterations)
        return out

    def info(self):
        q, r, p, u = C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
        F._raise(_lib().fwi_engine_info(self._h, C.byref(q), C.byref(r), C.byref(p), C.byref(u)))
        return dict(queued=q.value, running=r.value, pending=p.value, arena_used=int(u.value))

    def close(self):
        if self._h:
            rc = _lib().fwi_engine_destroy(self._h)
            self._h = C.c_void_p()
            F._raise(rc)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
