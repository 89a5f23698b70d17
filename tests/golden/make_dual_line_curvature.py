"""Writes dual_line_curvature.txt: where the second derivative of the ground energy E_0(g)
of the 3x3 unitary-gauge torus (Eq. (4), J = h = 1/2) along the dual line g = lambda is
smallest, next to the extremal point printed in the dual-line figure of Sec. V.

Calls only oracle/ (the Hamiltonian) and scipy's Lanczos solver; run from the
repository root:  python tests/golden/make_dual_line_curvature.py
"""
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import OracleLattice, Couplings  # noqa: E402
from oracle import ed  # noqa: E402

PRINTED = 0.1798   # caption of the dual-line second-derivative figure
J = H = 0.5


def ground_curve(lat, gs):
    """E_0(g) at lambda = g (H(g) = H(0, 0) + g (H(1, 1) - H(0, 0)))."""
    a = ed.hamiltonian(lat, Couplings(0.0, 0.0, J=J, h=H), 1.0)
    b = ed.hamiltonian(lat, Couplings(1.0, 1.0, J=J, h=H), 1.0) - a
    out, v0 = [], None
    for g in gs:
        w, v = spla.eigsh(a + g * b, k=1, which="SA", tol=1e-13, v0=v0, maxiter=100000)
        out.append(w[0])
        v0 = v[:, 0]
    return np.array(out)


def curvature_minimum(lat, lo, hi, h):
    gs = np.arange(lo, hi + 0.5 * h, h)
    e = ground_curve(lat, gs)
    d2 = (e[2:] - 2 * e[1:-1] + e[:-2]) / h ** 2
    i = int(np.argmin(d2[1:-1])) + 1
    y0, y1, y2 = d2[i - 1], d2[i], d2[i + 1]
    shift = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return gs[i + 1] + shift * h, y1 + 0.25 * (y0 - y2) * shift


def main():
    lat = OracleLattice(3, 3, True, "ug")
    g1, _ = curvature_minimum(lat, 0.10, 0.30, 0.005)
    g2, c2 = curvature_minimum(lat, g1 - 0.012, g1 + 0.012, 0.001)
    lines = ["# Minimum of d^2 E_0 / dg^2 along the dual line lambda = g on the 3x3 torus, unitary",
             "# gauge (Eq. (4)), J = h = 1/2: Lanczos ground energies on g steps of 0.005, then of",
             "# 0.001 around the coarse minimum, central second differences, parabola through the",
             "# smallest three.  Written by tests/golden/make_dual_line_curvature.py (oracle only).",
             "# The last column is the extremal point printed in the caption of the Sec. V dual-line",
             "# figure (adiabatic run from (0, 0.5) through (0.5, 0.5) to O).",
             "# columns: g_min(E_0)  d2E_0/dg2 at g_min  printed extremum",
             f"{g2:.5f}  {c2:.4f}  {PRINTED:.4f}"]
    print(lines[-1])
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "dual_line_curvature.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
