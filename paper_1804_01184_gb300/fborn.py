"""Binding of the frequency-domain Born calls of libfwi.so (Schemes I and II; C ABI in
include/fwi.h): ``fwi_fborn_workspace_bytes``, ``fwi_fborn_tables``, ``fwi_fborn_model``,
``fwi_fborn_gradient``, ``fwi_fborn_misfit``, ``fwi_fborn_hessian``.

Argument marshalling only: the Green tables, the Born contraction, the misfit, the gradient
and the Hessian all run in the library's kernels.  ``Acquisition`` holds one workspace with
the tables of a geometry and calls the rest against it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import fwi as F

LINEAR, NONLINEAR = 1, 2      # Scheme I (linear re-parameterization), Scheme II (exact)


class FGrid(C.Structure):
    """Mirror of ``fwi_fgrid``."""

    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("nf", C.c_int), ("dx", C.c_double), ("x0", C.c_double),
                ("z0", C.c_double), ("vp_o", C.c_double), ("rho_o", C.c_double)]


def make_fgrid(nx, nz, nf, dx, x0, z0, vp_o=2000.0, rho_o=2000.0) -> FGrid:
    return FGrid(int(nx), int(nz), int(nf), float(dx), float(x0), float(z0), float(vp_o), float(rho_o))


_bound = False


def lib():
    global _bound
    L = F.lib()
    if not _bound:
        gp, vp = C.POINTER(FGrid), C.c_void_p
        L.fwi_fborn_workspace_bytes.argtypes = [gp, C.c_int, C.c_int]
        L.fwi_fborn_workspace_bytes.restype = C.c_size_t
        L.fwi_fborn_tables.argtypes = [gp, vp, vp, vp, C.c_int, vp, C.c_int, vp, C.c_size_t, vp]
        L.fwi_fborn_model.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, C.c_int, vp, vp, vp]
        L.fwi_fborn_gradient.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.fwi_fborn_hessian.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]
        L.fwi_fborn_misfit.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
        L.fwi_fborn_status.argtypes = [gp, C.c_int, C.c_int, vp, vp]
        L.fwi_fborn_gradient_hessian.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, C.c_int, C.c_int,
                                                 vp, vp, vp, vp, vp]
        _bound = True
    return L


def fwi_fborn_workspace_bytes(fg: FGrid, ns: int, nr: int) -> int:
    n = lib().fwi_fborn_workspace_bytes(C.byref(fg), int(ns), int(nr))
    if n == 0:
        raise F.FwiError(-1, "invalid frequency-domain grid or sizes")
    return int(n)


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _complex_dev(t):
    """Contiguous complex64 CUDA tensor (from numpy or torch)."""
    if not torch.is_tensor(t):
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(t, np.complex64)))
    return t.to("cuda").to(torch.complex64).contiguous()


class Acquisition:
    """One acquisition (grid, frequencies, spectrum, sources, receivers) and its workspace of
    Green tables; fwi_fborn_tables runs on construction."""

    def __init__(self, fg: FGrid, freqs, spectrum, src_xy, rec_xy, stream=None):
        self.fg = fg
        self.freqs = _host(freqs, np.float64)
        spec = np.asarray(spectrum, np.complex64).reshape(-1)
        self.spec = np.ascontiguousarray(np.stack([spec.real, spec.imag], axis=1).astype(np.float32))
        self.src = _host(src_xy, np.float32).reshape(-1, 2)
        self.rec = _host(rec_xy, np.float32).reshape(-1, 2)
        self.ns, self.nr = self.src.shape[0], self.rec.shape[0]
        if self.freqs.shape[0] != fg.nf or self.spec.shape[0] != fg.nf:
            raise F.FwiError(-1, "freqs and spectrum must hold nf values")
        n = fwi_fborn_workspace_bytes(fg, self.ns, self.nr)
        self.work = torch.empty(n, dtype=torch.uint8, device="cuda")
        F._raise(lib().fwi_fborn_tables(C.byref(fg), self.freqs.ctypes.data_as(C.c_void_p),
                                        self.spec.ctypes.data_as(C.c_void_p), self.src.ctypes.data_as(C.c_void_p),
                                        self.ns, self.rec.ctypes.data_as(C.c_void_p), self.nr,
                                        F._ptr(self.work), n, F._stream(stream)))

    @property
    def shape(self):
        return (self.fg.nz, self.fg.nx)

    def model(self, pz, xi_a, xi_b, scheme=NONLINEAR, incident=True, out=None, stream=None):
        """Born data [nf][ns][nr] complex64 (fwi_fborn_model)."""
        xa, xb = F._dev(xi_a), F._dev(xi_b)
        if out is None:
            out = torch.empty((self.fg.nf, self.ns, self.nr), dtype=torch.complex64, device="cuda")
        F._raise(lib().fwi_fborn_model(C.byref(self.fg), self.ns, self.nr, int(scheme), int(pz), F._ptr(xa),
                                       F._ptr(xb), int(bool(incident)), F._ptr(self.work), F._ptr(out),
                                       F._stream(stream)))
        return out

    def gradient(self, pz, xi_a, xi_b, data_obs, scheme=LINEAR, misfit=None, grad=None, stream=None):
        """(misfit [1] float64, gradient [2][nz][nx] float64) (fwi_fborn_gradient)."""
        xa, xb, q = F._dev(xi_a), F._dev(xi_b), _complex_dev(data_obs)
        if misfit is None:
            misfit = torch.empty(1, dtype=torch.float64, device="cuda")
        if grad is None:
            grad = torch.empty((2,) + self.shape, dtype=torch.float64, device="cuda")
        F._raise(lib().fwi_fborn_gradient(C.byref(self.fg), self.ns, self.nr, int(scheme), int(pz), F._ptr(xa),
                                          F._ptr(xb), F._ptr(q), F._ptr(self.work), F._ptr(misfit), F._ptr(grad),
                                          F._stream(stream)))
        return misfit, grad

    def gradient_hessian(self, pz, xi_a, xi_b, data_obs, jx, jz, scheme=LINEAR, misfit=None, grad=None, H=None,
                         stream=None):
        """(misfit [1], gradient [2][nz][nx], Hessian terms [2][2][nz][nx] of node (jx, jz)), all
        float64, from one pass over the tables (fwi_fborn_gradient_hessian)."""
        xa, xb, q = F._dev(xi_a), F._dev(xi_b), _complex_dev(data_obs)
        if misfit is None:
            misfit = torch.empty(1, dtype=torch.float64, device="cuda")
        if grad is None:
            grad = torch.empty((2,) + self.shape, dtype=torch.float64, device="cuda")
        if H is None:
            H = torch.empty((2, 2) + self.shape, dtype=torch.float64, device="cuda")
        F._raise(lib().fwi_fborn_gradient_hessian(C.byref(self.fg), self.ns, self.nr, int(scheme), int(pz), F._ptr(xa),
                                                  F._ptr(xb), F._ptr(q), int(jx), int(jz), F._ptr(self.work),
                                                  F._ptr(misfit), F._ptr(grad), F._ptr(H), F._stream(stream)))
        return misfit, grad, H

    def misfit(self, pz, xi_a, xi_b, data_obs, scheme=LINEAR, out=None, stream=None):
        """Misfit [1] float64 alone (fwi_fborn_misfit)."""
        xa, xb, q = F._dev(xi_a), F._dev(xi_b), _complex_dev(data_obs)
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device="cuda")
        F._raise(lib().fwi_fborn_misfit(C.byref(self.fg), self.ns, self.nr, int(scheme), int(pz), F._ptr(xa),
                                        F._ptr(xb), F._ptr(q), F._ptr(self.work), F._ptr(out), F._stream(stream)))
        return out

    def hessian(self, pz, jx, jz, out=None, stream=None):
        """Scheme I Hessian terms H[a][b][nz][nx] for the fixed node (jx, jz)
        (fwi_fborn_hessian); H[:, :, jz, jx] is the reduced Hessian."""
        if out is None:
            out = torch.empty((2, 2) + self.shape, dtype=torch.float64, device="cuda")
        F._raise(lib().fwi_fborn_hessian(C.byref(self.fg), self.ns, self.nr, int(pz), int(jx), int(jz),
                                         F._ptr(self.work), F._ptr(out), F._stream(stream)))
        return out

    def status(self, stream=None):
        """Raises FwiError(FWI_ETIMEOUT) if a bounded device-side wait of the data contraction
        expired since the last check (fwi_fborn_status); synchronizes the stream."""
        F._raise(lib().fwi_fborn_status(C.byref(self.fg), self.ns, self.nr, F._ptr(self.work), F._stream(stream)))

    def reduced_hessian(self, pz, jx, jz, stream=None):
        return self.hessian(pz, jx, jz, stream=stream)[:, :, jz, jx]


def acquisition(w, stream=None) -> Acquisition:
    """The Acquisition of a frequency-domain workload (inputs.FreqWorkload)."""
    fg = make_fgrid(w.nx, w.nz, w.nf, w.dx, w.x0, w.z0, w.vp_o, w.rho_o)
    return Acquisition(fg, w.freqs, w.spectrum, w.src_xy, w.rec_xy, stream=stream)
