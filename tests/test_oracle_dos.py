"""Pins of the oracle's density of states of Z~ = -sum_l sigma^z_l (Sec. V)."""
from math import comb

import numpy as np
import pytest

import synth
from oracle import OracleLattice, Couplings
from oracle import core as O


@pytest.mark.parametrize("form", ["gh", "ug"])
def test_plus_state_is_binomial(form):
    lat = OracleLattice(2, 2, True, form)
    nl = len(lat.link_qubits)
    d = O.dos(O.plus_state(lat.n_qubits), lat)
    np.testing.assert_allclose(d, [comb(nl, k) / 2 ** nl for k in range(nl + 1)], atol=1e-15)


def test_basis_state_and_mean():
    lat = OracleLattice(2, 2, True, "gh")
    e = np.zeros(1 << lat.n_qubits, dtype=np.complex128)
    i = 0b101100110101
    e[i] = 1.0
    d = O.dos(e, lat)
    k = bin(i & sum(1 << q for q in lat.link_qubits)).count("1")
    assert d[k] == 1.0 and d.sum() == 1.0
    psi = O.evolve(lat, Couplings(0.6, 0.6), O.schedule_linear(3.0, 30), 0.1, 2)
    d = O.dos(psi, lat)
    nl = len(lat.link_qubits)
    mean = sum(d[k] * (2 * k - nl) for k in range(nl + 1))
    ztilde = -sum(O.expect_z(psi, 1 << q) for q in lat.link_qubits)
    assert mean == pytest.approx(ztilde, abs=1e-12)
    assert d.sum() == pytest.approx(1.0, abs=1e-12)
