"""Pins of the oracle's Trotter evolution.

* One step equals the product of exponentials of the dense group Hamiltonians
  (Eq. (7); Eq. (8) is exact because the summands of each group commute).
* The error against the exact piecewise-constant propagator scales as dt (first
  order) and dt^2 (second order).
* The per-step second-order error obeys the nested-commutator bound quoted in the
  Appendix (Childs et al.).
* Pure toric-code limit: every term commutes, so the Trotter product is exact and
  the B_p = +1 projected state (Sec. IV, Eq. (14)) is stationary.
* Invariants: norm, Gauss's law, lattice symmetry, 't Hooft loops at lambda = 0.
* The gauge-Higgs run restricted to tau = 0 equals the unitary-gauge run.
* Adiabatic endpoint energies respect the ground-energy (variational) bound.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import synth
from oracle import OracleLattice, Couplings
from oracle import core, ed


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("form", ["ug", "gh"])
def test_step_equals_group_exponentials(order, form):
    lat = OracleLattice(2, 2, True, form)
    c = Couplings(0.45, 0.8, J=0.7, h=1.2)
    s, dt = 0.63, 0.3
    psi0 = synth.random_state(lat.n_qubits, seed=5)
    psi = np.array(psi0)
    core.trotter_step(psi, lat, c, s, dt, order)
    hx, hz = ed.group_hamiltonians(lat, c, s)
    if order == 1:
        ref = spla.expm_multiply(-1j * dt * hz, spla.expm_multiply(-1j * dt * hx, psi0))
    else:
        ref = spla.expm_multiply(-0.5j * dt * hx, psi0)
        ref = spla.expm_multiply(-1j * dt * hz, ref)
        ref = spla.expm_multiply(-0.5j * dt * hx, ref)
    np.testing.assert_allclose(psi, ref, atol=1e-11)


def _global_error(lat, c, T, n_steps, order):
    s = core.schedule_linear(T, n_steps)
    dt = T / n_steps
    psi = core.evolve(lat, c, s, dt, order)
    ref = ed.exact_piecewise(lat, c, s, dt, core.plus_state(lat.n_qubits))
    return np.linalg.norm(psi - ref)


@pytest.mark.parametrize("form", ["ug", "gh"])
def test_trotter_order_slopes(form):
    lat = OracleLattice(2, 2, True, form)
    c = Couplings(0.6, 0.6)
    T = 2.0
    steps = [20, 40, 80, 160]
    for order, want in [(1, 1.0), (2, 2.0)]:
        errs = [_global_error(lat, c, T, n, order) for n in steps]
        slope = np.polyfit(np.log([T / n for n in steps]), np.log(errs), 1)[0]
        assert abs(slope - want) < 0.1, (order, errs, slope)


@pytest.mark.parametrize("s,dt", [(0.3, 0.2), (0.8, 0.1), (1.0, 0.05)])
def test_second_order_step_within_childs_bound(s, dt):
    """S_2 is assembled column by column from the oracle's own second-order step."""
    lat = OracleLattice(2, 2, True, "ug")
    c = Couplings(0.6, 0.6)
    dim = 1 << lat.n_qubits
    cols = []
    for j in range(dim):
        e = np.zeros(dim, dtype=np.complex128)
        e[j] = 1.0
        core.trotter_step(e, lat, c, s, dt, 2)
        cols.append(e)
    s2 = np.stack(cols, axis=1)
    err, bound = ed.second_order_step_error(lat, c, s, dt, s2=s2)
    err_dense, _ = ed.second_order_step_error(lat, c, s, dt)
    assert err == pytest.approx(err_dense, rel=1e-9)
    assert 0.0 < err <= bound


def _toric_projected(lat):
    """|+>^n projected onto B_p = +1 for every p (Eq. (14)), then normalised."""
    n = lat.n_qubits
    psi = core.plus_state(n)
    idx = np.arange(1 << n)
    for m in lat.z_plaquettes():
        par = np.array([bin(i & m).count("1") & 1 for i in idx])
        psi[par == 1] = 0.0
    return psi / np.linalg.norm(psi)


@pytest.mark.parametrize("order", [1, 2])
def test_toric_code_limit_is_exact(order):
    lat = OracleLattice(2, 2, True, "gh")
    c = Couplings(0.0, 0.0, J=1.0, h=1.0)
    psi0 = _toric_projected(lat)
    dt, n_steps = 0.7, 9                  # large dt: exact because all terms commute
    psi = core.evolve(lat, c, np.ones(n_steps), dt, order, psi0=psi0)
    Ns, Np = len(lat.vertices), len(lat.plaquettes)
    phase = np.exp(1j * (Ns + Np) * dt * n_steps)
    np.testing.assert_allclose(psi, phase * psi0, atol=1e-12)


def test_invariants_along_evolution():
    lat = OracleLattice(2, 2, True, "gh")
    c = Couplings(0.6, 0.6)
    T, n = 10.0, 100
    seen = []

    def cb(k, psi):
        if k % 25 == 24:
            obs = core.observables(psi, lat, c, 1.0)
            seen.append(obs)

    core.evolve(lat, c, core.schedule_linear(T, n), T / n, 1, callback=cb)
    for obs in seen:
        assert abs(obs["norm"] - 1.0) < 1e-12
        np.testing.assert_allclose(obs["gauss"], 1.0, atol=1e-12)
        np.testing.assert_allclose(obs["plaquettes"], obs["plaquettes"][0], atol=1e-12)
        xs = [obs["x"][q] for q in lat.link_qubits]
        np.testing.assert_allclose(xs, xs[0], atol=1e-12)


def test_thooft_loops_conserved_at_zero_lambda():
    lat = OracleLattice(3, 2, True, "ug")
    c = Couplings(0.7, 0.0)
    psi = core.evolve(lat, c, core.schedule_linear(3.0, 30), 0.1, 2)
    for m in lat.thooft():
        assert core.expect_x(psi, m) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_gauge_higgs_slice_equals_unitary_gauge(order):
    """psi_UG(sigma) = 2^{N_s/2} psi_GH(sigma, tau = 0) at every step."""
    gh = OracleLattice(3, 2, True, "gh")
    ug = OracleLattice(3, 2, True, "ug")
    c = Couplings(0.6, 0.6)
    T, n = 2.0, 10
    s = core.schedule_linear(T, n)
    psi_g = core.plus_state(gh.n_qubits)
    psi_u = core.plus_state(ug.n_qubits)
    nl, ns = ug.n_qubits, len(gh.vertices)
    for k in range(n):
        core.trotter_step(psi_g, gh, c, s[k], T / n, order)
        core.trotter_step(psi_u, ug, c, s[k], T / n, order)
        sl = psi_g[: 1 << nl] * 2 ** (ns / 2)
        np.testing.assert_allclose(sl, psi_u, atol=1e-12)


def test_adiabatic_endpoint_above_ground_energy():
    lat = OracleLattice(2, 2, True, "gh")
    for g, lam in [(0.2, 0.2), (1.2, 1.2)]:
        c = Couplings(g, lam)
        e0 = ed.ground_energy(lat, c, 1.0)[0]
        gaps = []
        for T in (5.0, 20.0):
            n = int(10 * T)
            psi = core.evolve(lat, c, core.schedule_linear(T, n), T / n, 2)
            e = core.energy(psi, lat, c, 1.0)
            e_ref = np.vdot(psi, ed.hamiltonian(lat, c, 1.0) @ psi).real
            assert e == pytest.approx(e_ref, abs=1e-11)
            assert e >= e0 - 1e-9
            gaps.append(e - e0)
        assert gaps[1] < gaps[0]
