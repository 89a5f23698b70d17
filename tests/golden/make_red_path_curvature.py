"""Writes red_path_curvature.txt: where the second derivative of the ground energy
E_0(g) of the 3x3 unitary-gauge torus (Eq. (4), J = h = 1/2) along lambda = r is
smallest, for the three broken red paths of the phase-diagram figure of Sec. V
(r = 0.05, 0.15, 0.25), next to the minima printed in that figure's caption.

Calls only oracle/ (the Hamiltonian) and scipy's Lanczos solver; run from the
repository root:  python tests/golden/make_red_path_curvature.py
"""
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import OracleLattice, Couplings  # noqa: E402
from oracle import ed  # noqa: E402

PRINTED = {0.05: 0.1920, 0.15: 0.1916, 0.25: 0.2489}   # caption of the second-derivative figure
J = H = 0.5


def ground_curve(lat, r, gs):
    """E_0(g) on the grid gs at lambda = r (H(g) = H(0, r) + g (H(1, r) - H(0, r)))."""
    a = ed.hamiltonian(lat, Couplings(0.0, r, J=J, h=H), 1.0)
    b = ed.hamiltonian(lat, Couplings(1.0, r, J=J, h=H), 1.0) - a
    out, v0 = [], None
    for g in gs:
        w, v = spla.eigsh(a + g * b, k=1, which="SA", tol=1e-13, v0=v0, maxiter=100000)
        out.append(w[0])
        v0 = v[:, 0]
    return np.array(out)


def curvature_minimum(lat, r, lo, hi, h):
    """g of the smallest central second difference of E_0 on [lo, hi] with step h,
    refined by a parabola through the smallest value and its neighbours."""
    gs = np.arange(lo, hi + 0.5 * h, h)
    e = ground_curve(lat, r, gs)
    d2 = (e[2:] - 2 * e[1:-1] + e[:-2]) / h ** 2
    i = int(np.argmin(d2[1:-1])) + 1
    y0, y1, y2 = d2[i - 1], d2[i], d2[i + 1]
    shift = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    return gs[i + 1] + shift * h, y1 + 0.25 * (y0 - y2) * shift


def main():
    lat = OracleLattice(3, 3, True, "ug")
    lines = ["# Minimum of d^2 E_0 / dg^2 along lambda = r on the 3x3 torus, unitary gauge (Eq. (4)),",
             "# J = h = 1/2: Lanczos ground energies on g steps of 0.005, then of 0.001 around the",
             "# coarse minimum, central second differences, parabola through the smallest three.",
             "# Written by tests/golden/make_red_path_curvature.py (oracle only).  The last column is",
             "# the minimum printed in the caption of the Sec. V second-derivative figure (adiabatic",
             "# runs along the broken red paths R(0.5, r) -> R'(0, r)).",
             "# columns: r  g_min(E_0)  d2E_0/dg2 at g_min  printed g_min"]
    for r in sorted(PRINTED):
        g1, _ = curvature_minimum(lat, r, 0.05, 0.45, 0.005)
        g2, c2 = curvature_minimum(lat, r, g1 - 0.012, g1 + 0.012, 0.001)
        lines.append(f"{r:.2f}  {g2:.5f}  {c2:.4f}  {PRINTED[r]:.4f}")
        print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "red_path_curvature.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
