"""Why the hysteresis energies of Sec. IV are read at one parameter point.

On an L x L torus the unitary-gauge Hamiltonian Eq. (4) with J = h is self-dual: a
Hadamard on every link together with the half-cell shift h(x, y) -> u(x+1, y),
u(x, y) -> h(x, y+1) of the link labels maps sigma^x <-> sigma^z, every star A_v to a
plaquette B_p and back, so H1(g, lambda) -> H1(lambda, g), and it maps psi_1' (Eq. (15))
to psi_1 (Eq. (14)).  The blue path P -> P' is the mirror image of P' -> P.  Hence the
energy of psi_1 carried O -> P -> P' and read at P' equals the energy of psi_1' carried
O -> P' -> P and read at P, for any protocol with exact propagators: comparing the two
path ends can never show the history dependence the paper reports.  The hysteresis
figure instead compares the two states at the same parameter point (its E lies at the
ground energy of P, its E' above it), i.e. E = <H1(P)> of psi_1 as prepared at P and
E' = <H1(P)> of psi_1' after it arrives at P; by the duality E' also equals the energy
of psi_1 after it arrives at P'.

These checks use the FP64 oracle on the 2 x 2 torus (8 link qubits, J = h = 1/2).
"""
import numpy as np
import scipy.linalg as sla

from oracle import OracleLattice, Couplings, mask_of
from oracle import core, ed

JH = 0.5


def _duality_permutation(lat):
    perm = {}
    for (x, y), q in lat.hlink.items():
        perm[q] = lat.ulink[((x + 1) % lat.Lx, y)]
    for (x, y), q in lat.ulink.items():
        perm[q] = lat.hlink[(x, (y + 1) % lat.Ly)]
    return perm


def _duality_matrix(lat, perm):
    n = lat.n_qubits
    dim = 1 << n
    idx = np.arange(dim)
    moved = np.zeros(dim, dtype=np.int64)
    for q, r in perm.items():
        moved |= ((idx >> q) & 1) << r
    P = np.zeros((dim, dim))
    P[moved, idx] = 1.0
    par = np.array([bin(i).count("1") & 1 for i in range(dim)])
    Hn = (1.0 - 2.0 * par[np.bitwise_and.outer(idx, idx)]) / np.sqrt(dim)
    return Hn @ P


def _segment(a, b, dg):
    a, b = np.asarray(a, float), np.asarray(b, float)
    n = int(round(float(np.max(np.abs(b - a))) / dg))
    return [Couplings(g, l, J=JH, h=JH) for g, l in (a + (b - a) * (k / n) for k in range(1, n + 1))]


def _exact_path(lat, psi, path, dt):
    for c in path:
        psi = sla.expm(-1j * dt * ed.dense(ed.hamiltonian(lat, c))) @ psi
    return psi


def _energy(lat, psi, c):
    return float(np.real(np.vdot(psi, ed.hamiltonian(lat, c) @ psi)))


def test_self_duality_of_the_torus():
    lat = OracleLattice(2, 2, True, "ug")
    perm = _duality_permutation(lat)
    assert sorted(perm.values()) == list(range(lat.n_qubits))
    plaq = {m for m in lat.z_plaquettes()}
    stars = {mask_of(s) for s in lat.stars}
    assert {mask_of([perm[q] for q in s]) for s in lat.stars} == plaq
    assert {mask_of([perm[q] for q in p]) for p in lat.plaquettes} == stars
    U = _duality_matrix(lat, perm)
    for g, lam in ((0.12, 0.0), (0.3, 0.07), (0.0, 0.5)):
        h = ed.dense(ed.hamiltonian(lat, Couplings(g, lam, J=JH, h=JH)))
        hd = ed.dense(ed.hamiltonian(lat, Couplings(lam, g, J=JH, h=JH)))
        np.testing.assert_allclose(U @ h @ U.conj().T, hd, atol=1e-12)
    psi1 = core.toric_state(lat, 0)
    psi1p = core.toric_state(lat, 1)
    assert abs(abs(np.vdot(psi1, U @ psi1p)) - 1.0) <= 1e-12


def test_path_end_energies_are_equal_by_duality():
    """E at the end of O -> P -> P' for psi_1 equals E' at the end of O -> P' -> P for
    psi_1' (exact propagators), while the energies of the two states at the same point
    P differ."""
    lat = OracleLattice(2, 2, True, "ug")
    p, dg, dt = 0.12, 0.004, 0.05
    P, Pp = (p, 0.0), (0.0, p)
    a = _exact_path(lat, core.toric_state(lat, 0), _segment((0, 0), P, dg), dt)
    e_a_at_P = _energy(lat, a, Couplings(*P, J=JH, h=JH))
    a = _exact_path(lat, a, _segment(P, Pp, dg), dt)
    e_a_at_Pp = _energy(lat, a, Couplings(*Pp, J=JH, h=JH))
    b = _exact_path(lat, core.toric_state(lat, 1), _segment((0, 0), Pp, dg), dt)
    b = _exact_path(lat, b, _segment(Pp, P, dg), dt)
    e_b_at_P = _energy(lat, b, Couplings(*P, J=JH, h=JH))
    assert abs(e_a_at_Pp - e_b_at_P) <= 1e-11                 # the end-to-end reading: E = E'
    assert abs(e_a_at_P - e_b_at_P) >= 1e-3                    # the same-point reading: E != E'
    # the Trotterised oracle (second order) keeps the end-to-end identity up to the
    # ordering of the two factor groups (dt = 0.02, the paper's step), far below the
    # printed |E - E'| = 0.00964
    at = core.evolve_path(lat, _segment((0, 0), P, dg) + _segment(P, Pp, dg), 0.02, 2,
                          psi0=core.toric_state(lat, 0))
    bt = core.evolve_path(lat, _segment((0, 0), Pp, dg) + _segment(Pp, P, dg), 0.02, 2,
                          psi0=core.toric_state(lat, 1))
    d = abs(_energy(lat, at, Couplings(*Pp, J=JH, h=JH)) - _energy(lat, bt, Couplings(*P, J=JH, h=JH)))
    assert d <= 1e-4, d
