"""Thin Python binding of libfwi.so (C ABI in include/fwi.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch supplies device memory (inputs, outputs and the scratch workspace) and streams.
The functions carry the C names: ``fwi_model``, ``fwi_born``, ``fwi_adjoint``,
``fwi_gradient`` (optionally weighted per trace), ``fwi_misfit``, ``fwi_workspace_bytes``,
``fwi_status``, ``fwi_model_noalloc``, ``fwi_status_noalloc``, ``fwi_set_tile``, ``fwi_set_checkpoint``,
``fwi_set_accumulation``, ``fwi_trace``.

There is no fallback: if libfwi.so has not been built (``paper_1804_01184_gb300.build``)
or no CUDA device is present, these functions raise.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import threading

import torch

from . import build as _build

VP_RHO, IP_RHO, VP_IP, K_RHO, INVK_INVRHO = range(5)
OP_MODEL, OP_BORN, OP_ADJOINT, OP_GRADIENT = range(4)
ERRORS = {0: "FWI_OK", -1: "FWI_EINVAL", -2: "FWI_ECFL", -3: "FWI_ENOMEM", -4: "FWI_ETIMEOUT", -5: "FWI_ECUDA"}


class FwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    """Mirror of ``fwi_grid``."""

    _fields_ = [
        ("nx", C.c_int), ("nz", C.c_int), ("sponge", C.c_int), ("order", C.c_int), ("nt", C.c_int),
        ("dx", C.c_double), ("dt", C.c_double), ("vp_o", C.c_double), ("rho_o", C.c_double),
        ("sponge_v", C.c_double), ("sponge_R", C.c_double),
    ]


class _Sources(C.Structure):
    _fields_ = [("ns", C.c_int), ("xy", C.c_void_p), ("wavelet", C.c_void_p)]


class _Receivers(C.Structure):
    _fields_ = [("nr", C.c_int), ("xy", C.c_void_p)]


def make_grid(nx, nz, dx, dt, nt, order=8, sponge=40, vp_o=2000.0, rho_o=2000.0, sponge_v=None,
              sponge_R=1e-3) -> Grid:
    return Grid(int(nx), int(nz), int(sponge), int(order), int(nt), float(dx), float(dt), float(vp_o),
                float(rho_o), float(vp_o if sponge_v is None else sponge_v), float(sponge_R))


_lib = None
_lock = threading.Lock()


def _open(path):
    """Loads the library at `path` and binds every single-job entry point."""
    L = C.CDLL(path)
    gp, vp, dp = C.POINTER(Grid), C.c_void_p, C.c_void_p
    sp, rp = C.POINTER(_Sources), C.POINTER(_Receivers)
    L.fwi_workspace_bytes.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_size_t]
    L.fwi_workspace_bytes.restype = C.c_size_t
    L.fwi_model.argtypes = [gp, C.c_int, vp, vp, sp, rp, vp, vp, C.c_size_t, vp]
    L.fwi_born.argtypes = [gp, C.c_int, vp, vp, vp, vp, sp, rp, vp, vp, C.c_size_t, vp]
    L.fwi_adjoint.argtypes = [gp, C.c_int, vp, vp, sp, rp, vp, dp, vp, C.c_size_t, vp]
    L.fwi_gradient.argtypes = [gp, C.c_int, vp, vp, sp, rp, vp, dp, dp, vp, C.c_size_t, vp]
    L.fwi_status.argtypes = [vp, vp]
    L.fwi_misfit.argtypes = [vp, vp, C.c_longlong, vp, vp]
    L.fwi_misfit_weighted.argtypes = [vp, vp, C.c_longlong, C.c_int, vp, vp, vp]
    L.fwi_gradient_weighted.argtypes = [gp, C.c_int, vp, vp, sp, rp, vp, vp, dp, dp, vp, C.c_size_t, vp]
    L.fwi_last_error.restype = C.c_char_p
    L.fwi_launch_count.restype = C.c_longlong
    L.fwi_set_tile.argtypes = [C.c_int, C.c_int]
    L.fwi_set_checkpoint.argtypes = [C.c_int]
    L.fwi_set_accumulation.argtypes = [C.c_int]
    L.fwi_trace.argtypes = [C.c_int]
    L.fwi_trace_report.argtypes = [C.c_char_p, C.c_size_t]
    L.fwi_model_noalloc.argtypes = [gp, C.c_int, vp, vp, sp, rp, vp, vp]
    L.fwi_status_noalloc.argtypes = [vp]
    L.fwi_profile.argtypes = [C.c_int]
    L.fwi_profile_report.argtypes = [C.c_char_p, C.c_size_t]
    return L


def lib():
    """The loaded libfwi.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfwi.so is not built ({path}); run paper_1804_01184_gb300.build.build()")
            _lib = _open(path)
    return _lib


@contextlib.contextmanager
def library(path):
    """Runs the single-job calls made inside the block on the library at `path` -- e.g. the
    bounds-checked debug build, build.LIB_CHECKED -- then returns to the default one."""
    global _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built")
    with _lock:
        prev = _lib
        _lib = _open(path)
    try:
        yield _lib
    finally:
        with _lock:
            _lib = prev


def _raise(rc):
    if rc != 0:
        raise FwiError(rc, lib().fwi_last_error().decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev(t, dtype=torch.float32):
    """Contiguous CUDA tensor of dtype (copies host arrays / numpy to the current device)."""
    if not torch.is_tensor(t):
        t = torch.as_tensor(t)
    if not t.is_cuda:
        t = t.to("cuda", non_blocking=False)
    return t.to(dtype).contiguous()


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class _OnStream:
    """Orders a library call on a caller-given stream after the current stream (where the
    binding converted and copied the inputs) and, after the call, ties every tensor the call
    reads or writes to that stream, so the caching allocator does not reuse their memory
    before the library's kernels are done with it.  No-op for the current stream."""

    def __init__(self, stream):
        cur = torch.cuda.current_stream()
        self.stream = stream if stream is not None and stream != cur else None
        if self.stream is not None:
            self.stream.wait_stream(cur)

    def keep(self, *tensors):
        if self.stream is None:
            return
        for t in tensors:
            if isinstance(t, (tuple, list)):
                self.keep(*t)
            elif torch.is_tensor(t) and t.is_cuda:
                t.record_stream(self.stream)


def fwi_workspace_bytes(grid: Grid, ns: int, nr: int, op: int, budget_bytes: int = 0) -> int:
    n = lib().fwi_workspace_bytes(C.byref(grid), int(ns), int(nr), int(op), int(budget_bytes))
    if n == 0:
        raise FwiError(-1, "invalid grid or sizes")
    return int(n)


def default_budget(device=None) -> int:
    """Workspace budget: 80 % of the free device memory."""
    free, _ = torch.cuda.mem_get_info(device)
    return int(free * 0.8)


def workspace(grid: Grid, ns: int, nr: int, op: int, budget_bytes: int | None = None) -> torch.Tensor:
    """A device buffer of the bytes the library plans for `op` within `budget_bytes`."""
    budget = default_budget() if budget_bytes is None else int(budget_bytes)
    n = fwi_workspace_bytes(grid, ns, nr, op, budget)
    return torch.empty(n, dtype=torch.uint8, device="cuda")


def fwi_status(work: torch.Tensor, stream=None):
    _raise(lib().fwi_status(_ptr(work), _stream(stream)))


def fwi_set_tile(tz: int = 0, variant: int = 0):
    """Launch-shape override for plans made afterwards (0, 0 = built-in defaults)."""
    _raise(lib().fwi_set_tile(int(tz), int(variant)))


def fwi_set_checkpoint(every: int = 0):
    """Checkpoint interval for gradient plans made afterwards (0 = the planner chooses)."""
    _raise(lib().fwi_set_checkpoint(int(every)))


def fwi_set_accumulation(steps: int = 0):
    """Adjoint steps per FP32 gradient-accumulation chunk for plans made afterwards (0 = 64)."""
    _raise(lib().fwi_set_accumulation(int(steps)))


def fwi_trace(enable: bool = True):
    """NVTX phase ranges on (True) or off for later operations on any thread."""
    _raise(lib().fwi_trace(int(bool(enable))))


def trace_report() -> dict:
    """Ranges opened per phase since the last report ({phase: count}); resets the counts."""
    buf = C.create_string_buffer(1 << 12)
    lib().fwi_trace_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt = line.rsplit(" ", 1)
        out[name] = int(cnt)
    return out


def launch_count() -> int:
    return int(lib().fwi_launch_count())


def _acq(src_xy, wavelet, rec_xy):
    s, w, r = _dev(src_xy).reshape(-1, 2), _dev(wavelet).reshape(-1), _dev(rec_xy).reshape(-1, 2)
    return (s, w, r), _Sources(s.shape[0], s.data_ptr(), w.data_ptr()), _Receivers(r.shape[0], r.data_ptr())


def fwi_model(grid: Grid, pz: int, xi_a, xi_b, src_xy, wavelet, rec_xy, traces=None, work=None,
              stream=None, check=True) -> torch.Tensor:
    """Forward traces [ns][nr][nt] float32 (see fwi_model in include/fwi.h)."""
    a, b = _dev(xi_a), _dev(xi_b)
    keep, S, R = _acq(src_xy, wavelet, rec_xy)
    if traces is None:
        traces = torch.empty((S.ns, R.nr, grid.nt), dtype=torch.float32, device="cuda")
    if work is None:
        work = workspace(grid, S.ns, R.nr, OP_MODEL)
    on = _OnStream(stream)
    _raise(lib().fwi_model(C.byref(grid), int(pz), _ptr(a), _ptr(b), C.byref(S), C.byref(R), _ptr(traces),
                           _ptr(work), work.numel(), _stream(stream)))
    on.keep(a, b, keep, traces, work)
    if check:
        fwi_status(work, stream)
    return traces


def fwi_model_noalloc(grid: Grid, pz: int, xi_a, xi_b, src_xy, wavelet, rec_xy, traces=None,
                      stream=None, check=True) -> torch.Tensor:
    """fwi_model on the library's built-in scratch, for callers that cannot allocate device
    memory (see fwi_model_noalloc in include/fwi.h: size limit, first-call set-up, sharing).
    check: wait for the stream and raise the data-dependent errors the call recorded
    (fwi_status_noalloc)."""
    a, b = _dev(xi_a), _dev(xi_b)
    keep, S, R = _acq(src_xy, wavelet, rec_xy)
    if traces is None:
        traces = torch.empty((S.ns, R.nr, grid.nt), dtype=torch.float32, device="cuda")
    on = _OnStream(stream)
    _raise(lib().fwi_model_noalloc(C.byref(grid), int(pz), _ptr(a), _ptr(b), C.byref(S), C.byref(R),
                                   _ptr(traces), _stream(stream)))
    on.keep(a, b, keep, traces)
    if check:
        fwi_status_noalloc(stream)
    return traces


def fwi_status_noalloc(stream=None):
    """Raises the data-dependent error the last fwi_model_noalloc call on this device recorded."""
    _raise(lib().fwi_status_noalloc(_stream(stream)))


def fwi_born(grid: Grid, pz: int, xi_a, xi_b, dxi_a, dxi_b, src_xy, wavelet, rec_xy, dtraces=None,
             work=None, stream=None, check=True) -> torch.Tensor:
    """Born traces [ns][nr][nt] float32 for the contrast perturbation (dxi_a, dxi_b)."""
    a, b, da, db = _dev(xi_a), _dev(xi_b), _dev(dxi_a), _dev(dxi_b)
    keep, S, R = _acq(src_xy, wavelet, rec_xy)
    if dtraces is None:
        dtraces = torch.empty((S.ns, R.nr, grid.nt), dtype=torch.float32, device="cuda")
    if work is None:
        work = workspace(grid, S.ns, R.nr, OP_BORN)
    on = _OnStream(stream)
    _raise(lib().fwi_born(C.byref(grid), int(pz), _ptr(a), _ptr(b), _ptr(da), _ptr(db), C.byref(S),
                          C.byref(R), _ptr(dtraces), _ptr(work), work.numel(), _stream(stream)))
    on.keep(a, b, da, db, keep, dtraces, work)
    if check:
        fwi_status(work, stream)
    return dtraces


def fwi_adjoint(grid: Grid, pz: int, xi_a, xi_b, src_xy, wavelet, rec_xy, residual, grads=None, work=None,
                stream=None, check=True) -> torch.Tensor:
    """Gradient of sum(residual * traces) for all five parameterizations: [5][2][nz][nx] float64."""
    a, b, res = _dev(xi_a), _dev(xi_b), _dev(residual)
    keep, S, R = _acq(src_xy, wavelet, rec_xy)
    if grads is None:
        grads = torch.empty((5, 2, grid.nz, grid.nx), dtype=torch.float64, device="cuda")
    if work is None:
        work = workspace(grid, S.ns, R.nr, OP_ADJOINT)
    on = _OnStream(stream)
    _raise(lib().fwi_adjoint(C.byref(grid), int(pz), _ptr(a), _ptr(b), C.byref(S), C.byref(R), _ptr(res),
                             _ptr(grads), _ptr(work), work.numel(), _stream(stream)))
    on.keep(a, b, res, keep, grads, work)
    if check:
        fwi_status(work, stream)
    return grads


def fwi_gradient(grid: Grid, pz: int, xi_a, xi_b, src_xy, wavelet, rec_xy, data, misfit=None, grads=None,
                 work=None, stream=None, check=True, weights=None):
    """Misfit (device float64 scalar tensor) and gradients [5][2][nz][nx] float64.  weights:
    optional [ns][nr] per-trace weights (fwi_gradient_weighted)."""
    a, b, d = _dev(xi_a), _dev(xi_b), _dev(data)
    keep, S, R = _acq(src_xy, wavelet, rec_xy)
    if grads is None:
        grads = torch.empty((5, 2, grid.nz, grid.nx), dtype=torch.float64, device="cuda")
    if misfit is None:
        misfit = torch.empty((), dtype=torch.float64, device="cuda")
    if work is None:
        work = workspace(grid, S.ns, R.nr, OP_GRADIENT)
    wt = _dev(weights) if weights is not None else None
    if wt is not None and wt.numel() != S.ns * R.nr:
        raise FwiError(-1, "weights must hold ns x nr values")
    on = _OnStream(stream)
    if wt is None:
        _raise(lib().fwi_gradient(C.byref(grid), int(pz), _ptr(a), _ptr(b), C.byref(S), C.byref(R), _ptr(d),
                                  _ptr(misfit), _ptr(grads), _ptr(work), work.numel(), _stream(stream)))
    else:
        _raise(lib().fwi_gradient_weighted(C.byref(grid), int(pz), _ptr(a), _ptr(b), C.byref(S), C.byref(R),
                                           _ptr(d), _ptr(wt), _ptr(misfit), _ptr(grads), _ptr(work), work.numel(),
                                           _stream(stream)))
    on.keep(a, b, d, wt, keep, misfit, grads, work)
    if check:
        fwi_status(work, stream)
    return misfit, grads


def fwi_misfit(traces, data, misfit=None, stream=None, weights=None, nt=None) -> torch.Tensor:
    """J = 1/2 sum (traces - data)^2 (float64 device scalar tensor), in the library's kernel;
    with weights (one per trace of nt samples), J = 1/2 sum_t w_t sum_n (...)^2."""
    t, d = _dev(traces), _dev(data)
    if t.numel() != d.numel():
        raise FwiError(-1, "traces and data differ in size")
    if misfit is None:
        misfit = torch.empty((), dtype=torch.float64, device="cuda")
    wt = _dev(weights) if weights is not None else None
    if wt is not None and (nt is None or wt.numel() * nt != t.numel()):
        raise FwiError(-1, "weights x nt must cover the traces")
    on = _OnStream(stream)
    if wt is None:
        _raise(lib().fwi_misfit(_ptr(t), _ptr(d), t.numel(), _ptr(misfit), _stream(stream)))
    else:
        _raise(lib().fwi_misfit_weighted(_ptr(t), _ptr(d), wt.numel(), int(nt), _ptr(wt), _ptr(misfit),
                                         _stream(stream)))
    on.keep(t, d, wt, misfit)
    return misfit
