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
