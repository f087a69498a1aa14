"""FP64 oracle of the frequency-domain Born modelling of Schemes I and II (test infrastructure).

TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA frequency-domain Born kernels
are checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the CUDA path (numpy + scipy only).

What it computes (Sec. "Modelling and Inversion", Sec. "Point-scatterer Analysis"):

- the reference Green function G_o of the homogeneous operator w^2/K_o + div (1/rho_o) grad,
  from the 2-D Hankel function of the first kind;
- the modelling vector W(x, w; x_r, x_s) of the Born approximation (eqn:param_born): the
  bulk-modulus term w^2/K_o G_o(x_r, x) G_o(x, x_s) and the density term
  -(1/rho_o) grad G_o(x_r, x) . grad G_o(x, x_s);
- Born data p = S(w) [G_o(x_r, x_s) + sum_x W(x)^T xi_{1/K,1/rho}(x) dx^2] (eqn:param_pfreq1),
  with the contrasts of parameterization pz mapped to (xi_{1/K}, xi_{1/rho}) linearly
  (Scheme I, Table 3) or exactly (Scheme II, Table 2);
- the misfit J = 1/2 sum_{w >= 0} sum_{s,r} |p - q|^2 and its gradient in the contrasts of
  pz (chain rule through the map);
- the Hessian of J for Scheme I (eqn:param_Hker and the terms H_(a,i),(b,j) of
  eqn:param_Hfull with x_j fixed), whose 2 x 2 block at x_i = x_j is the reduced Hessian.

Readings where the paper is silent or loose (each one also listed in the design notes):

- F1: G_o = (i rho_o / 4) H_0^(1)(k r), k = w / c_o, for the e^{-iwt} convention; this sign
  makes the Lippmann-Schwinger equation as printed (a plus sign before the scattering
  integrals) exact.  W holds two factors of G_o and the residual cancels the incident field,
  so the misfit, its gradient and the Hessians do not depend on that sign.
- F2: the model integral is a sum over the nodes of a regular grid times dx^2.
- F3: the source spectrum S(w) and the frequencies are inputs (the tests use the Ricker's
  own spectrum at f_k = k df, k = 1 .. nf; the DC term, where a Ricker has no energy, is
  left out).
- F4: the Hessian of the real misfit in real contrasts is the REAL part of the paper's
  sum S S* W* W^T; for Scheme I (linear map, Born data linear in the contrasts) it is the
  exact second derivative of J.
- F5: Scheme I's linear map is the linearization at zero contrast of the exact map; for the
  impedance row that is xi_Ip = -(xi_{1/K} + xi_{1/rho}) / 2, not the printed
  xi_{1/rho} - xi_{1/K} / 2 of Table 3 (a misprint: it disagrees with Table 2).

Parameterizations (Table 1): 0 vp-rho (A), 1 Ip-rho (B), 2 vp-Ip (C), 3 K-rho (D),
4 1/K-1/rho (E).  Arrays are [nz][nx] (x fastest); node (i, j) sits at (x0 + i dx, z0 + j dx).
"""
from __future__ import annotations

import numpy as np
from scipy.special import hankel1

LINEAR, NONLINEAR = 1, 2


class FGrid:
    """The model grid of the frequency-domain modelling and its homogeneous reference."""

    def __init__(self, nx, nz, dx, x0, z0, vp_o=2000.0, rho_o=2000.0):
        self.nx, self.nz, self.dx, self.x0, self.z0 = int(nx), int(nz), float(dx), float(x0), float(z0)
        self.vp_o, self.rho_o = float(vp_o), float(rho_o)

    @property
    def K_o(self):
        return self.rho_o * self.vp_o ** 2

    def nodes(self):
        """[N][2] coordinates of the nodes, x fastest."""
        x = self.x0 + self.dx * np.arange(self.nx)
        z = self.z0 + self.dx * np.arange(self.nz)
        X, Z = np.meshgrid(x, z)
        return np.stack([X.ravel(), Z.ravel()], axis=1)


def green(fg, f, r):
    """G_o at distance r and its radial derivative dG_o/dr at frequency f (Hz) (reading F1):
    G_o = (i rho_o/4) H_0^(1)(k r), dG_o/dr = -(i rho_o k/4) H_1^(1)(k r) (H_0' = -H_1)."""
    k = 2.0 * np.pi * f / fg.vp_o
    r = np.asarray(r, np.float64)
    G = 1j * fg.rho_o / 4.0 * hankel1(0, k * r)
    dG = -1j * fg.rho_o * k / 4.0 * hankel1(1, k * r)
    return G, dG


def _point_fields(fg, f, pts, X):
    """G_o(x, p), grad_x G_o(x, p) for points p [np][2] and nodes X [N][2]:
    ([np][N], [np][N][2])."""
    d = X[None, :, :] - np.asarray(pts, np.float64)[:, None, :]
    r = np.sqrt((d ** 2).sum(-1))
    G, dG = green(fg, f, r)
    return G, dG[..., None] * (d / r[..., None])


def modelling_vectors(fg, f, src, rec):
    """W(x, w; x_r, x_s) of eqn:param_born at frequency f for every source s, receiver r and
    node x: complex [ns][nr][N][2] (component 0: xi_{1/K}, 1: xi_{1/rho})."""
    X = fg.nodes()
    w = 2.0 * np.pi * f
    Gs, gGs = _point_fields(fg, f, src, X)
    Gr, gGr = _point_fields(fg, f, rec, X)
    W1 = (w * w / fg.K_o) * Gr[None, :, :] * Gs[:, None, :]
    W2 = -(1.0 / fg.rho_o) * np.einsum("rnd,snd->srn", gGr, gGs)
    return np.stack([W1, W2], axis=-1)


def incident(fg, f, src, rec):
    """G_o(x_r, w; x_s): complex [ns][nr]."""
    d = np.asarray(rec, np.float64)[None, :, :] - np.asarray(src, np.float64)[:, None, :]
    return green(fg, f, np.sqrt((d ** 2).sum(-1)))[0]


# ---------------------------------------------------------------- re-parameterizations

def to_inverse_contrasts(pz, a, b, scheme):
    """(xi_{1/K}, xi_{1/rho}) of contrasts (a, b) of parameterization pz (Table 1), exactly
    (Scheme II: the relations behind Table 2) or linearized at zero contrast (Scheme I, the
    inverse of Table 3; reading F5 for the impedance)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if scheme == LINEAR:
        L = linear_jacobian(pz)
        return L[0, 0] * a + L[0, 1] * b, L[1, 0] * a + L[1, 1] * b
    if pz == 0:     # K = rho vp^2
        return 1.0 / ((1 + b) * (1 + a) ** 2) - 1.0, 1.0 / (1 + b) - 1.0
    if pz == 1:     # K = Ip^2 / rho
        return (1 + b) / (1 + a) ** 2 - 1.0, 1.0 / (1 + b) - 1.0
    if pz == 2:     # K = Ip vp, rho = Ip / vp
        return 1.0 / ((1 + a) * (1 + b)) - 1.0, (1 + a) / (1 + b) - 1.0
    if pz == 3:
        return 1.0 / (1 + a) - 1.0, 1.0 / (1 + b) - 1.0
    return a.copy(), b.copy()


def linear_jacobian(pz):
    """d(xi_{1/K}, xi_{1/rho}) / d(xi_a, xi_b) at zero contrast: the Scheme I map."""
    return {0: np.array([[-2.0, -1.0], [0.0, -1.0]]),
            1: np.array([[-2.0, 1.0], [0.0, -1.0]]),
            2: np.array([[-1.0, -1.0], [1.0, -1.0]]),
            3: np.array([[-1.0, 0.0], [0.0, -1.0]]),
            4: np.eye(2)}[pz]


def jacobian(pz, a, b, scheme):
    """Per-node Jacobian d(xi_{1/K}, xi_{1/rho}) / d(xi_a, xi_b): [2][2][...]."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    one, zero = np.ones_like(a), np.zeros_like(a)
    if scheme == LINEAR:
        L = linear_jacobian(pz)
        return np.array([[L[0, 0] * one, L[0, 1] * one], [L[1, 0] * one, L[1, 1] * one]])
    A, B = 1 + a, 1 + b
    if pz == 0:
        return np.array([[-2.0 / (B * A ** 3), -1.0 / (B * B * A * A)], [zero, -1.0 / (B * B)]])
    if pz == 1:
        return np.array([[-2.0 * B / A ** 3, 1.0 / (A * A)], [zero, -1.0 / (B * B)]])
    if pz == 2:
        return np.array([[-1.0 / (A * A * B), -1.0 / (A * B * B)], [1.0 / B, -A / (B * B)]])
    if pz == 3:
        return np.array([[-1.0 / (A * A), zero], [zero, -1.0 / (B * B)]])
    return np.array([[one, zero], [zero, one]])


# ---------------------------------------------------------------- modelling and inversion

def model(fg, freqs, spectrum, src, rec, pz, xi_a, xi_b, scheme, with_incident=True):
    """Born data p[f][s][r] (complex) of eqn:param_pfreq1 for the contrasts (xi_a, xi_b)
    of parameterization pz, mapped by `scheme`."""
    e1, e2 = to_inverse_contrasts(pz, np.ravel(xi_a), np.ravel(xi_b), scheme)
    xi = np.stack([e1, e2], axis=-1)
    out = []
    for f, S in zip(freqs, np.asarray(spectrum, np.complex128)):
        W = modelling_vectors(fg, f, src, rec)
        p = np.einsum("srnc,nc->sr", W, xi) * fg.dx ** 2
        if with_incident:
            p = p + incident(fg, f, src, rec)
        out.append(S * p)
    return np.array(out)


def misfit(p, q):
    """J = 1/2 sum_{w, s, r} |p - q|^2."""
    return 0.5 * float(np.sum(np.abs(np.asarray(p) - np.asarray(q)) ** 2))


def gradient(fg, freqs, spectrum, src, rec, pz, xi_a, xi_b, q, scheme):
    """(J, dJ/dxi_a, dJ/dxi_b) at contrasts (xi_a, xi_b) of pz against observed data q:
    dJ/dxi_{1/K,1/rho}(x) = Re sum conj(p - q) S W(x) dx^2, then the chain rule through the
    map of `scheme` (Sec. "Modelling and Inversion")."""
    p = model(fg, freqs, spectrum, src, rec, pz, xi_a, xi_b, scheme)
    R = p - q
    gE = np.zeros((fg.nz * fg.nx, 2))
    for k, (f, S) in enumerate(zip(freqs, np.asarray(spectrum, np.complex128))):
        W = modelling_vectors(fg, f, src, rec)
        gE += np.real(np.einsum("sr,srnc->nc", np.conj(R[k]), S * W)) * fg.dx ** 2
    Jm = jacobian(pz, np.ravel(xi_a), np.ravel(xi_b), scheme)
    ga = Jm[0, 0] * gE[:, 0] + Jm[1, 0] * gE[:, 1]
    gb = Jm[0, 1] * gE[:, 0] + Jm[1, 1] * gE[:, 1]
    shape = (fg.nz, fg.nx)
    return misfit(p, q), ga.reshape(shape), gb.reshape(shape)


def hessian_column(fg, freqs, spectrum, src, rec, pz, j):
    """Scheme I Hessian terms H_(a,i),(b,j) = d^2 J / d xi_a(x_i) d xi_b(x_j) for the fixed
    node j (flat index) and every node i: [2][2][nz][nx] (reading F4: the real part of
    sum |S|^2 sum_{s,r} conj(W_a(x_i)) W_b(x_j) dx^4, mapped by the Scheme I Jacobian)."""
    N = fg.nz * fg.nx
    HE = np.zeros((2, 2, N))
    for f, S in zip(freqs, np.asarray(spectrum, np.complex128)):
        W = modelling_vectors(fg, f, src, rec)
        HE += (abs(S) ** 2) * np.real(np.einsum("srna,srb->abn", np.conj(W), W[:, :, j, :])) * fg.dx ** 4
    L = linear_jacobian(pz)
    H = np.einsum("ca,cdn,db->abn", L, HE, L)
    return H.reshape(2, 2, fg.nz, fg.nx)


def reduced_hessian(fg, freqs, spectrum, src, rec, pz, j):
    """The 2 x 2 reduced Hessian of eqn:param_Hker at node j (Scheme I)."""
    iz, ix = divmod(j, fg.nx)
    return hessian_column(fg, freqs, spectrum, src, rec, pz, j)[:, :, iz, ix]
