"""Pins of the oracle's lattice and Hamiltonian against structural facts of the model.

* Every link bounds two plaquettes (torus) and joins two vertices (Sec. II).
* Stars and plaquettes share 0 or 2 links, so [A_v, B_p] = 0 (toric code).
* prod_p B_p = prod_v A_v = 1 on a torus.
* Gauss's law: Q_v = tau^x_v A^x_v commutes with H (Eq. (1), Eq. (3)).
* The toric code (g = lambda = 0) on a torus has E_0 = -(N_v + N_p) with a
  four-fold degenerate ground space (Sec. IV: psi_1..psi_4 are degenerate).
* The gauge-Higgs form restricted to Q_v = +1 has the spectrum of the
  unitary-gauge form (the mapping stated before Eq. (4)).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import OracleLattice, Couplings, mask_of
from oracle import ed


@pytest.mark.parametrize("L", [(2, 2), (3, 3), (4, 4), (3, 2)])
def test_periodic_counts_and_incidence(L):
    lat = OracleLattice(L[0], L[1], True, "gh")
    N = L[0] * L[1]
    assert lat.n_links == 2 * N and lat.n_sites == N and lat.n_qubits == 3 * N
    assert len(lat.plaquettes) == N and len(lat.stars) == N and len(lat.bonds) == 2 * N
    links = lat.link_qubits
    assert sorted(links) == list(range(2 * N))
    for q in links:
        assert sum(q in p for p in lat.plaquettes) == 2
        assert sum(q in s for s in lat.stars) == 2
    for p in lat.plaquettes:
        assert len(set(p)) == 4
        for s in lat.stars:
            assert len(set(p) & set(s)) in (0, 2)
    acc = 0
    for m in lat.z_plaquettes():
        acc ^= m
    assert acc == 0
    acc = 0
    for s in lat.stars:
        acc ^= mask_of(s)
    assert acc == 0
    ug = OracleLattice(L[0], L[1], True, "ug")
    assert ug.n_qubits == 2 * N


def test_open_3x2_unitary_gauge_has_17_links():
    lat = OracleLattice(3, 2, False, "ug")
    assert lat.n_qubits == 17
    assert len(lat.plaquettes) == 6 and len(lat.stars) == 12
    assert sorted(len(s) for s in lat.stars) == [2] * 4 + [3] * 6 + [4] * 2
    for q in lat.link_qubits:
        assert sum(q in s for s in lat.stars) == 2
        assert sum(q in p for p in lat.plaquettes) in (1, 2)
    for p in lat.plaquettes:
        for s in lat.stars:
            assert len(set(p) & set(s)) in (0, 2)


def test_bond_and_gauss_geometry():
    lat = OracleLattice(3, 3, True, "gh")
    for (tj, sl, tk), (q, a, b) in zip(lat.bonds, lat.links):
        assert sl == q and tj == lat.site[a] and tk == lat.site[b]
    for mq, v, s in zip(lat.gauss(), lat.vertices, lat.stars):
        assert mq == mask_of([lat.site[v]] + s)
        # Q_v commutes with every Z term: even overlap
        for m in lat.z_plaquettes() + lat.z_second():
            assert bin(mq & m).count("1") % 2 == 0


def test_gauss_law_commutes_with_hamiltonian():
    lat = OracleLattice(2, 2, True, "gh")
    c = Couplings(0.37, 0.81, J=0.9, h=1.3)
    H = ed.hamiltonian(lat, c, 0.6)
    for m in lat.gauss():
        Q = ed.xstring_matrix(lat.n_qubits, m)
        comm = (H @ Q - Q @ H)
        assert abs(comm).max() < 1e-12


@pytest.mark.parametrize("L", [(2, 2), (3, 2)])
def test_toric_code_ground_space(L):
    lat = OracleLattice(L[0], L[1], True, "ug")
    c = Couplings(0.0, 0.0, J=1.0, h=1.0)
    w = ed.ground_energy(lat, c, 1.0, k=6)
    N = L[0] * L[1]
    np.testing.assert_allclose(w[:4], -2.0 * N, atol=1e-9)
    assert w[4] > -2.0 * N + 1.0


def test_gauge_higgs_sector_equals_unitary_gauge():
    gh = OracleLattice(2, 2, True, "gh")
    ug = OracleLattice(2, 2, True, "ug")
    for g, lam in [(0.2, 0.2), (0.6, 0.6), (1.2, 0.3)]:
        c = Couplings(g, lam)
        a = ed.ground_energy(gh, c, 1.0, k=4)
        b = ed.ground_energy(ug, c, 1.0, k=4)
        np.testing.assert_allclose(a, b, atol=1e-9)


def test_group_hamiltonians_commute_internally():
    """Summands inside each group commute (the remark after Eq. (8))."""
    lat = OracleLattice(2, 2, True, "ug")
    n = lat.n_qubits
    xs = [ed.xstring_matrix(n, 1 << q) for q in lat.link_qubits]
    xs += [ed.xstring_matrix(n, m) for m in lat.x_strings()]
    for a in xs:
        for b in xs:
            assert abs(a @ b - b @ a).max() < 1e-14
