"""Pins of the oracle's toric-code initial states and parameter paths (Sec. III-IV).

* psi_1 (Eq. (14)) and psi_1' (Eq. (15)) are toric-code ground states: B_p = A_v = +1.
* psi_1 is a +1 eigenstate of both 't Hooft loops, psi_1' of both Wilson loops.
* Sec. IV: psi_1' = (psi_1 + psi_2 + psi_3 + psi_4) / 2 with psi_2 = W_1 psi_1,
  psi_3 = W_2 psi_1, psi_4 = W_1 W_2 psi_1.
* Their energy at g = lambda = 0 (J = h = 1/2) is -(N_v + N_p)/2.
* A path with constant couplings equals the s = 1 evolution.
"""
import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O


@pytest.mark.parametrize("L", [(2, 2), (3, 2)])
def test_toric_states(L):
    lat = OracleLattice(L[0], L[1], True, "ug")
    p1 = O.toric_state(lat, 0)
    p1d = O.toric_state(lat, 1)
    for psi in (p1, p1d):
        assert O.norm2(psi) == pytest.approx(1.0, abs=1e-13)
        for m in lat.z_plaquettes():
            assert O.expect_z(psi, m) == pytest.approx(1.0, abs=1e-12)
        for st in lat.stars:
            assert O.expect_x(psi, sum(1 << q for q in st)) == pytest.approx(1.0, abs=1e-12)
        e = O.energy(psi, lat, Couplings(0.0, 0.0, J=0.5, h=0.5), 1.0)
        assert e == pytest.approx(-(len(lat.stars) + len(lat.plaquettes)) / 2, abs=1e-12)
    for m in lat.thooft():
        assert O.expect_x(p1, m) == pytest.approx(1.0, abs=1e-12)
    for m in lat.wilson():
        assert O.expect_z(p1d, m) == pytest.approx(1.0, abs=1e-12)
    # psi_1' = (psi_1 + W_1 psi_1 + W_2 psi_1 + W_1 W_2 psi_1) / 2
    w1, w2 = lat.wilson()
    idx = np.arange(p1.size)
    sign = lambda m: 1.0 - 2.0 * np.array([bin(i & m).count("1") & 1 for i in idx])
    combo = 0.5 * (p1 + sign(w1) * p1 + sign(w2) * p1 + sign(w1) * sign(w2) * p1)
    np.testing.assert_allclose(combo, p1d, atol=1e-12)


def test_constant_path_equals_s_one_evolution():
    lat = OracleLattice(2, 2, True, "ug")
    c = Couplings(0.3, 0.2, J=0.5, h=0.5)
    a = O.evolve_path(lat, [c] * 7, 0.1, 2, psi0=O.toric_state(lat, 0))
    b = O.evolve(lat, c, np.ones(7), 0.1, 2, psi0=O.toric_state(lat, 0))
    np.testing.assert_allclose(a, b, atol=1e-14)
