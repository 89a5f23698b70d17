"""Parameter paths of the adiabatic protocol (Sec. III, Sec. IV, Sec. VI).

The model is the unitary-gauge form, Eq. (4), with J = h = 1/2 on the (g, lambda) plane.
A path is a list of per-step coupling records; step k evolves under H1 with those
couplings (qs_evolve_path).  Along a straight segment the couplings change by a fixed
amount per step in the leading coordinate, g_n = n * dg as in the error analysis.

  O = (0, 0)        toric-code point: psi_1 (Eq. (14)) or psi_1' (Eq. (15))
  P = (p, 0)        on the g axis
  P' = (0, p)       on the lambda axis
  R = (p, r), R' = (0, r)   red path  P -> R -> R'
  blue path         P -> P' (straight line)
"""
from __future__ import annotations

import numpy as np


def segment(a, b, dg: float, J: float = 0.5, h: float = 0.5):
    """Couplings (g, lambda, J, h) of the steps from point a to point b, excluding a."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = int(round(float(np.max(np.abs(b - a))) / dg))
    if n == 0:
        return []
    return [(float(g), float(l), J, h) for g, l in (a + (b - a) * (k / n) for k in range(1, n + 1))]


def prepare(p: float, dg: float, axis: str = "g", J: float = 0.5, h: float = 0.5):
    """From O along one axis to (p, 0) (axis g) or (0, p) (axis lambda)."""
    end = (p, 0.0) if axis == "g" else (0.0, p)
    return segment((0.0, 0.0), end, dg, J, h)


def blue(p: float, dg: float, reverse: bool = False, J: float = 0.5, h: float = 0.5):
    """P(p, 0) -> P'(0, p), or P' -> P when reverse."""
    a, b = ((p, 0.0), (0.0, p)) if not reverse else ((0.0, p), (p, 0.0))
    return segment(a, b, dg, J, h)


def red(p: float, r: float, dg: float, J: float = 0.5, h: float = 0.5):
    """P(p, 0) -> R(p, r) -> R'(0, r)."""
    return segment((p, 0.0), (p, r), dg, J, h) + segment((p, r), (0.0, r), dg, J, h)


def run_path(sim, path, dt: float, order: int = 2, measure_every: int = 0):
    """Evolve the bound state along `path`; if measure_every > 0 return the energies
    <H1(path[k])> after every measure_every steps (and at the end) with their couplings."""
    if measure_every <= 0:
        if path:
            sim.evolve_path(path, dt, order)
        return []
    out = []
    for k0 in range(0, len(path), measure_every):
        piece = path[k0:k0 + measure_every]
        sim.evolve_path(piece, dt, order)
        c = piece[-1]
        out.append((c, float(sim.energy([c])[0])))
    return out
