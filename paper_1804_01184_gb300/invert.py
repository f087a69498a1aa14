"""Steepest-descent inversion (Sec. "Modelling and Inversion": gradient-based minimisation of
the least-squares data misfit), used to compare how fast each parameterization converges.

Each iteration takes the misfit gradient, steps along the negative gradient, and chooses the
step by a line search over trial models.  Two modelling back ends:

- ``Inversion`` (Scheme III): the gradient from fwi_gradient (forward, adjoint, chain rule);
  the trial models run together as jobs of the batching engine, their misfits reduced by
  fwi_misfit.
- ``BornInversion`` (Schemes I and II): the frequency-domain Born path of fborn.Acquisition
  (fwi_fborn_gradient, fwi_fborn_misfit), under the linear or the exact map.

- Known shape g (scatterers (i), (ii), (iv), (v)): the unknowns are the two contrasts (a, b)
  of (xi_a, xi_b) = (a g, b g); their gradient is the field gradient projected on g,
  dJ/da = <dJ/dxi_a, g>.
- Unknown shape (scatterers (iii), (vi), (vii)): the unknowns are the contrast fields
  themselves.

The paper does not say which line search it used; here (a reading): trial steps
alpha_k = alpha * 2^k, k = -3 .. 4, the best one kept and alpha re-centred on it for the next
iteration; when no trial lowers the misfit the step is refined by shrinking alpha by 16 (at
most three times) before the iteration gives up.
"""
from __future__ import annotations

import numpy as np
import torch

from . import engine as E
from . import fwi as F


class _SteepestDescent:
    """The descent loop shared by the back ends: they supply fields(m), gradient(m) ->
    (J, g) and misfits(list of m) -> numpy misfits; self.g is the known shape or None."""

    alpha = None

    # model of a parameter vector: (a, b) scalars with a known shape, else two fields
    def fields(self, m):
        if self.g is not None:
            return self.g * float(m[0]), self.g * float(m[1])
        return m[0], m[1]

    def project(self, J, ga, gb):
        """(J, gradient in the parameter vector): projected on the shape when it is known."""
        if self.g is not None:
            g64 = self.g.double()
            return J, (torch.sum(ga * g64).item(), torch.sum(gb * g64).item())
        return J, (ga.float(), gb.float())

    @staticmethod
    def step(m, d, alpha):
        return (m[0] + alpha * d[0], m[1] + alpha * d[1])

    def run(self, m0, iters=10, trials=8):
        """Returns (final parameters, misfit history [J_0, J_1, ...])."""
        m = m0
        J, g = self.gradient(m)
        hist = [J]
        for _ in range(iters):
            d = (-g[0], -g[1])
            if self.alpha is None:   # first step: a 5 % change of the largest contrast
                gmax = max(abs(d[0]), abs(d[1])) if self.g is not None else \
                    max(d[0].abs().max().item(), d[1].abs().max().item())
                self.alpha = 0.05 / max(gmax, 1e-30)
            best = None
            for _shrink in range(4):
                alphas = [self.alpha * 2.0 ** k for k in range(-3, trials - 3)]
                Js = self.misfits([self.step(m, d, a) for a in alphas])
                k = int(np.argmin(Js))
                if Js[k] < J:
                    best = (alphas[k], Js[k])
                    break
                self.alpha /= 16.0
            if best is None:
                break
            self.alpha = best[0]
            m = self.step(m, d, best[0])
            J, g = self.gradient(m)
            hist.append(J)
        return m, hist


class Inversion(_SteepestDescent):
    def __init__(self, w, pz, data, shape=None, arena_bytes=1 << 30, weights=None):
        self.w, self.pz, self.shape = w, pz, shape
        self.grid = F.make_grid(**w.grid_kwargs())
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        self.src, self.rec, self.wav = d(w.src_xy), d(w.rec_xy), d(w.wavelet)
        self.data = F._dev(data)
        self.g = d(shape) if shape is not None else None
        self.weights = d(weights) if weights is not None else None   # [ns][nr] trace weights
        self.work = F.workspace(self.grid, w.ns, w.nr, F.OP_GRADIENT)
        self.engine = E.Engine(arena_bytes)
        self.alpha = None

    def gradient(self, m):
        xa, xb = self.fields(m)
        J, G = F.fwi_gradient(self.grid, self.pz, xa, xb, self.src, self.wav, self.rec, self.data, work=self.work,
                              weights=self.weights)
        return self.project(J.item(), G[self.pz, 0], G[self.pz, 1])

    def misfits(self, models):
        """Misfit of each model (a list of parameter vectors), all as jobs of one engine run."""
        out = torch.empty(len(models), dtype=torch.float64, device="cuda")
        self.engine.stream.wait_stream(torch.cuda.current_stream())   # the trial models are ready
        tick = {}
        with torch.cuda.stream(self.engine.stream):
            for k, m in enumerate(models):
                xa, xb = self.fields(m)
                tick[self.engine.submit_model(self.grid, self.pz, xa, xb, self.src, self.wav, self.rec,
                                              work_budget=1 << 28)] = k
        flat = self.data.reshape(-1)
        while tick:
            for r in self.engine.run(64):
                F.fwi_misfit(r.traces.reshape(-1), flat, misfit=out[tick.pop(r.ticket)], stream=self.engine.stream,
                             weights=self.weights, nt=self.w.nt)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    def close(self):
        self.engine.close()


class BornInversion(_SteepestDescent):
    """Schemes I/II: steepest descent on the frequency-domain Born misfit of parameterization
    pz against observed data (complex [nf][ns][nr]); scheme FB.LINEAR (Scheme I) or
    FB.NONLINEAR (Scheme II).  shape: the known shape g (then the unknowns are its two
    contrasts), or None (the unknowns are the two contrast fields)."""

    def __init__(self, acq, pz, data, scheme, shape=None):
        self.acq, self.pz, self.scheme = acq, pz, scheme
        self.data = data if torch.is_tensor(data) else torch.from_numpy(np.asarray(data, np.complex64)).cuda()
        self.g = torch.from_numpy(np.ascontiguousarray(shape)).cuda() if shape is not None else None
        self.alpha = None

    def gradient(self, m):
        xa, xb = self.fields(m)
        J, G = self.acq.gradient(self.pz, xa, xb, self.data, scheme=self.scheme)
        return self.project(J.item(), G[0], G[1])

    def misfits(self, models):
        out = torch.empty(len(models), dtype=torch.float64, device="cuda")
        for k, m in enumerate(models):
            xa, xb = self.fields(m)
            self.acq.misfit(self.pz, xa, xb, self.data, scheme=self.scheme, out=out[k:k + 1])
        return out.cpu().numpy()

    def close(self):
        pass
