"""The oracle's model against energies printed in the paper.

The hysteresis figure of Sec. IV prints adiabatic energies on the 3x3 torus (unitary
gauge, J = h = 1/2, tests/golden/hysteresis_endpoints.txt).  An adiabatically prepared
state cannot lie below the ground energy of its Hamiltonian, and a slow path keeps it
close: the Lanczos ground energy of the oracle's Hamiltonian at the path end points
(g, lambda) = (p, 0) and (0, p) (equal by the self-duality of Eq. (4)) must be at most
the printed energies and within 0.02 of them.  This fixes the lattice (18 links, 9
stars, 9 plaquettes) and the normalisation of Eq. (4).
"""
import os

import pytest

from oracle import OracleLattice, Couplings
from oracle import ed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hysteresis_endpoints.txt")


def test_printed_hysteresis_energies_sit_just_above_the_ground_energy():
    lat = OracleLattice(3, 3, True, "ug")
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for p, e, e2 in rows:
        p, e, e2 = float(p), float(e), float(e2)
        e0_a = ed.ground_energy(lat, Couplings(p, 0.0, J=0.5, h=0.5), 1.0)[0]
        e0_b = ed.ground_energy(lat, Couplings(0.0, p, J=0.5, h=0.5), 1.0)[0]
        assert e0_a == pytest.approx(e0_b, abs=1e-9)          # self-duality g <-> lambda
        for printed in (e, e2):
            assert e0_a <= printed + 1e-9
            assert printed - e0_a < 0.02
    # toric-code point: E_0 = -(N_v + N_p) / 2 = -9
    assert ed.ground_energy(lat, Couplings(0.0, 0.0, J=0.5, h=0.5), 1.0)[0] == pytest.approx(-9.0, abs=1e-9)


CURVATURE = os.path.join(os.path.dirname(__file__), "golden", "red_path_curvature.txt")


def test_ground_energy_curvature_minima_match_the_printed_phase_transition_points():
    """Sec. V locates the transitions along the broken red paths (lambda = r, g from 0.5
    down to 0) at the minima of d^2E/dg^2: g = 0.1920, 0.1916, 0.2489 for r = 0.05, 0.15,
    0.25.  The oracle's Hamiltonian gives those minima for its ground energy E_0(g)
    within 0.003 (golden file written by tests/golden/make_red_path_curvature.py); the
    tabulated curvature at r = 0.25 is recomputed here from three Lanczos energies on
    each side of the tabulated minimum and in its centre."""
    import numpy as np
    rows = [[float(x) for x in l.split()] for l in open(CURVATURE) if l.strip() and not l.startswith("#")]
    assert [r[0] for r in rows] == [0.05, 0.15, 0.25]
    for r, g_min, d2, printed in rows:
        assert abs(g_min - printed) <= 0.003
        assert d2 < -80.0
    lat = OracleLattice(3, 3, True, "ug")
    r, g_min, d2, _ = rows[2]
    h = 0.001

    def curv(g):
        e = [ed.ground_energy(lat, Couplings(g + d, r, J=0.5, h=0.5), 1.0)[0] for d in (-h, 0.0, h)]
        return (e[0] - 2 * e[1] + e[2]) / h ** 2

    c0 = curv(g_min)
    assert abs(c0 - d2) <= 0.5
    assert curv(g_min - 0.004) > c0 and curv(g_min + 0.004) > c0


DUAL = os.path.join(os.path.dirname(__file__), "golden", "dual_line_curvature.txt")


def test_ground_energy_curvature_on_the_dual_line_matches_the_printed_extremum():
    """Sec. V finds an extremal point of d^2E/dg^2 on the dual line lambda = g at g_3 =
    0.1798, inside the deconfined phase.  The oracle's ground energy E_0(g) along the same
    line has its curvature minimum within 0.003 of it (golden file written by
    tests/golden/make_dual_line_curvature.py); the tabulated curvature is recomputed from
    three Lanczos energies, and is lower than 0.004 to either side."""
    rows = [[float(x) for x in l.split()] for l in open(DUAL) if l.strip() and not l.startswith("#")]
    (g_min, d2, printed), = rows
    assert abs(g_min - printed) <= 0.003
    lat = OracleLattice(3, 3, True, "ug")
    h = 0.001

    def curv(g):
        e = [ed.ground_energy(lat, Couplings(g + d, g + d, J=0.5, h=0.5), 1.0)[0] for d in (-h, 0.0, h)]
        return (e[0] - 2 * e[1] + e[2]) / h ** 2

    c0 = curv(g_min)
    assert abs(c0 - d2) <= 0.5
    assert curv(g_min - 0.004) > c0 and curv(g_min + 0.004) > c0
