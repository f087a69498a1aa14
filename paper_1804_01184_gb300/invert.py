"""Steepest-descent inversion (Sec. "Modelling and Inversion": gradient-based minimisation of
the least-squares data misfit), used to compare how fast each parameterization converges.

Each iteration takes the misfit gradient from fwi_gradient (forward, adjoint, chain rule),
steps along the negative gradient, and chooses the step by a line search whose trial models
all run together as jobs of the batching engine (their misfits reduced by fwi_misfit).

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


class Inversion:
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

    # model of a parameter vector: (a, b) scalars with a known shape, else two fields
    def fields(self, m):
        if self.g is not None:
            return self.g * float(m[0]), self.g * float(m[1])
        return m[0], m[1]

    def gradient(self, m):
        xa, xb = self.fields(m)
        J, G = F.fwi_gradient(self.grid, self.pz, xa, xb, self.src, self.wav, self.rec, self.data, work=self.work,
                              weights=self.weights)
        ga, gb = G[self.pz, 0], G[self.pz, 1]
        if self.g is not None:
            g64 = self.g.double()
            return J.item(), (torch.sum(ga * g64).item(), torch.sum(gb * g64).item())
        return J.item(), (ga.float(), gb.float())

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

    def close(self):
        self.engine.close()
