"""FP64 CPU oracle for the Scheme III hot path of arXiv:1804.01184 (test infrastructure).

TEST INFRASTRUCTURE ONLY: this package is the slow, plain reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path and imports nothing from
the ``paper_1804_01184_gb300`` package.

The arithmetic lives in ``fwi_oracle.c`` (plain C, FP64); this module compiles it with gcc
(``build()``) and wraps it with ctypes.  Every function cites the passage of the paper it
follows in the C source.  Parity pins (tests/test_oracle_*.py) fix it against the analytic
2-D Green function, reciprocity, discrete energy, the adjoint dot-product test, Taylor
tests and brute-force finite differences.

Parameterizations (Table 1): 0 = vp-rho (A), 1 = Ip-rho (B), 2 = vp-Ip (C), 3 = K-rho (D),
4 = 1/K-1/rho (E).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

PARAMETERIZATIONS = ("vp-rho", "Ip-rho", "vp-Ip", "K-rho", "1/K-1/rho")


class Grid(C.Structure):
    """Mirror of ``og_grid`` in fwi_oracle.c."""

    _fields_ = [
        ("nx", C.c_int), ("nz", C.c_int), ("sponge", C.c_int), ("order", C.c_int),
        ("nt", C.c_int), ("dx", C.c_double), ("dt", C.c_double), ("vp_o", C.c_double),
        ("rho_o", C.c_double), ("sponge_v", C.c_double), ("sponge_R", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile fwi_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(Grid)
            L.oracle_coefficients.argtypes = [C.c_int, dp]
            L.oracle_apply_d.argtypes = [C.c_int, dp, dp, C.c_int, C.c_int, C.c_double]
            L.oracle_forward_map.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
            L.oracle_chain_rule.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_model_build.argtypes = [gp, C.c_int, dp, dp, dp, dp, dp, dp]
            L.oracle_sponge_profile.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                                C.c_double, C.c_int, dp]
            L.oracle_sponge_profile.restype = None
            L.oracle_weights.argtypes = [gp, C.c_double, C.c_double, C.POINTER(C.c_long), dp]
            L.oracle_model.argtypes = [gp, C.c_int, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp]
            L.oracle_energy.argtypes = [gp, C.c_int, dp, dp, dp, dp, dp]
            L.oracle_born.argtypes = [gp, C.c_int, dp, dp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp]
            L.oracle_adjoint.argtypes = [gp, C.c_int, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp, dp, dp]
            L.oracle_gradient.argtypes = [gp, C.c_int, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp, dp, dp, dp]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def make_grid(nx, nz, dx, dt, nt, order=8, sponge=40, vp_o=2000.0, rho_o=2000.0,
              sponge_v=None, sponge_R=1e-3) -> Grid:
    return Grid(int(nx), int(nz), int(sponge), int(order), int(nt), float(dx), float(dt),
                float(vp_o), float(rho_o), float(vp_o if sponge_v is None else sponge_v),
                float(sponge_R))


def coefficients(order):
    c = np.zeros(4)
    _, cp = _d(c)
    c_arr = (C.c_double * 4)()
    M = lib().oracle_coefficients(order, c_arr)
    _check(0 if M > 0 else -1, "coefficients")
    return np.array(c_arr[:M])


def apply_d(f, order, minus, dx=1.0):
    f, fp = _d(f)
    out, op = _d(np.zeros_like(f))
    _check(lib().oracle_apply_d(f.size, fp, op, order, int(minus), dx), "apply_d")
    return out


def forward_map(pz, a, b, vp_o=2000.0, rho_o=2000.0):
    K, rho = C.c_double(), C.c_double()
    _check(lib().oracle_forward_map(pz, a, b, vp_o, rho_o, C.byref(K), C.byref(rho)), "forward_map")
    return K.value, rho.value


def chain_rule(vp_o, rho_o, K, rho, gK, grho):
    K, Kp = _d(K)
    rho, rp = _d(rho)
    gK, gKp = _d(gK)
    grho, grp = _d(grho)
    out, op = _d(np.zeros((5, 2) + K.shape))
    _check(lib().oracle_chain_rule(vp_o, rho_o, K.size, Kp, rp, gKp, grp, op), "chain_rule")
    return out


def model_build(g: Grid, pz, xi_a, xi_b):
    Nx, Nz = g.nx + 2 * g.sponge, g.nz + 2 * g.sponge
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    outs = [np.zeros((Nz, Nx)) for _ in range(4)]
    ptrs = [_d(o)[1] for o in outs]
    _check(lib().oracle_model_build(C.byref(g), pz, ap, bp, *ptrs), "model_build")
    return tuple(outs)  # K, rho, bx, bz


def sponge_profile(n, S, dx, dt, v, R, half):
    d = np.zeros(n + 2 * S)
    _, dp = _d(d)
    arr = (C.c_double * d.size)()
    lib().oracle_sponge_profile(n, S, dx, dt, v, R, int(half), arr)
    return np.array(arr[:])


def weights(g: Grid, x, z):
    idx = (C.c_long * 4)()
    w = (C.c_double * 4)()
    _check(lib().oracle_weights(C.byref(g), float(x), float(z), idx, w), "weights")
    return np.array(idx[:]), np.array(w[:])


def model(g: Grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy):
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    s, sp = _d(np.reshape(src_xy, (-1, 2)))
    w, wp = _d(wavelet)
    r, rp = _d(np.reshape(rec_xy, (-1, 2)))
    ns, nr = s.shape[0], r.shape[0]
    out, op = _d(np.zeros((ns, nr, g.nt)))
    _check(lib().oracle_model(C.byref(g), pz, ap, bp, ns, sp, wp, nr, rp, op), "model")
    return out


def energy(g: Grid, pz, xi_a, xi_b, src_xy, wavelet):
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    s, sp = _d(np.reshape(src_xy, (-1, 2))[:1])
    w, wp = _d(wavelet)
    out, op = _d(np.zeros(g.nt))
    _check(lib().oracle_energy(C.byref(g), pz, ap, bp, sp, wp, op), "energy")
    return out


def born(g: Grid, pz, xi_a, xi_b, dxi_a, dxi_b, src_xy, wavelet, rec_xy):
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    da, dap = _d(dxi_a)
    db, dbp = _d(dxi_b)
    s, sp = _d(np.reshape(src_xy, (-1, 2)))
    w, wp = _d(wavelet)
    r, rp = _d(np.reshape(rec_xy, (-1, 2)))
    ns, nr = s.shape[0], r.shape[0]
    out, op = _d(np.zeros((ns, nr, g.nt)))
    _check(lib().oracle_born(C.byref(g), pz, ap, bp, dap, dbp, ns, sp, wp, nr, rp, op), "born")
    return out


def adjoint(g: Grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, residual, with_krho=False):
    """Gradient of sum(residual * traces): returns grads [5][2][nz][nx] (and [2][nz][nx] for K, rho)."""
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    s, sp = _d(np.reshape(src_xy, (-1, 2)))
    w, wp = _d(wavelet)
    r, rp = _d(np.reshape(rec_xy, (-1, 2)))
    res, resp = _d(residual)
    ns, nr = s.shape[0], r.shape[0]
    assert res.shape == (ns, nr, g.nt)
    grads, gp = _d(np.zeros((5, 2, g.nz, g.nx)))
    kr, krp = _d(np.zeros((2, g.nz, g.nx)))
    _check(lib().oracle_adjoint(C.byref(g), pz, ap, bp, ns, sp, wp, nr, rp, resp, gp, krp), "adjoint")
    return (grads, kr) if with_krho else grads


def gradient(g: Grid, pz, xi_a, xi_b, src_xy, wavelet, rec_xy, data, with_krho=False):
    """Misfit J = 1/2 sum (d_mod - d_obs)^2 and its gradient for all five parameterizations."""
    a, ap = _d(xi_a)
    b, bp = _d(xi_b)
    s, sp = _d(np.reshape(src_xy, (-1, 2)))
    w, wp = _d(wavelet)
    r, rp = _d(np.reshape(rec_xy, (-1, 2)))
    d, dp_ = _d(data)
    ns, nr = s.shape[0], r.shape[0]
    assert d.shape == (ns, nr, g.nt)
    J = C.c_double()
    grads, gp = _d(np.zeros((5, 2, g.nz, g.nx)))
    kr, krp = _d(np.zeros((2, g.nz, g.nx)))
    _check(lib().oracle_gradient(C.byref(g), pz, ap, bp, ns, sp, wp, nr, rp, dp_, C.byref(J), gp, krp),
           "gradient")
    return (J.value, grads, kr) if with_krho else (J.value, grads)
