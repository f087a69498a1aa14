"""Diffraction patterns (Sec. "Diffraction-pattern Analysis"): the energy a point scatterer with
a unit contrast in ONE parameter of a parameterization scatters towards each receiver, as a
function of the scattering angle -- the angle between the incident direction (source to
scatterer) and the scattered one (scatterer to receiver).

The scattered data come from the frequency-domain Born path (``fborn.Acquisition.model``,
incident field off) under the linear map of Scheme I, so the pattern of parameter a of
parameterization pz is that of the modelling vector W taken through the map's column a:
in 1/K-1/rho the bulk-modulus term radiates the same in every direction and the density term
as cos^2 of the scattering angle.  The energy is summed over the acquisition's frequencies
(weighted by the source spectrum).
"""
from __future__ import annotations

import numpy as np
import torch

from . import fborn as FBN


def scattering_angles(src_xy, rec_xy, x0):
    """[ns][nr] scattering angles in degrees (0: forward scattering) at point x0."""
    s = np.asarray(src_xy, np.float64).reshape(-1, 2)
    r = np.asarray(rec_xy, np.float64).reshape(-1, 2)
    inc = np.asarray(x0, np.float64) - s
    sca = r - np.asarray(x0, np.float64)
    inc /= np.linalg.norm(inc, axis=1, keepdims=True)
    sca /= np.linalg.norm(sca, axis=1, keepdims=True)
    return np.degrees(np.arccos(np.clip(inc @ sca.T, -1.0, 1.0)))


def diffraction_pattern(acq, pz, param, jx, jz, stream=None):
    """Scattered energy sum_f |p_sr|^2 [ns][nr] (float64 numpy) of a unit contrast of
    parameter `param` (0: first, 1: second of parameterization pz) at node (jx, jz)."""
    nz, nx = acq.shape
    xa = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    xb = torch.zeros_like(xa)
    (xa if param == 0 else xb)[jz, jx] = 1.0
    d = acq.model(pz, xa, xb, scheme=FBN.LINEAR, incident=False, stream=stream)
    return (d.abs().double() ** 2).sum(0).cpu().numpy()


def pattern_summary(energy, angles, at=(0.0, 45.0, 90.0, 135.0, 180.0)):
    """Energy relative to its maximum at the receivers nearest the given scattering angles
    (averaged over the sources)."""
    e = energy / energy.max()
    out = {}
    for a in at:
        vals = [e[s, int(np.argmin(np.abs(angles[s] - a)))] for s in range(e.shape[0])]
        out[f"{a:g}"] = round(float(np.mean(vals)), 4)
    return out


def cos2(angles):
    """cos^2 of scattering angles in degrees: the shape of the density term's pattern."""
    return np.cos(np.radians(angles)) ** 2

