"""Pins of the oracle's forward-mode gradients and of the error-bound arithmetic.

* dE/da_m and dF/da_m from forward tangents agree with central finite
  differences of the oracle's own evolution (a different algorithm).
* The closed-form bound of Sec. VI reproduces Table I (tests/golden), and the
  step-by-step sum of the Appendix's per-step bound agrees with the closed form.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import OracleLattice, Couplings
from oracle import core, bound

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_trotter_bound.txt")


@pytest.mark.parametrize("target", ["energy", "fidelity"])
def test_forward_tangents_match_finite_differences(target):
    lat = OracleLattice(2, 2, True, "gh")
    c = Couplings(0.6, 0.6)
    T, n, M = 4.0, 40, 4
    a = synth.fourier_coeffs(M, seed=3, std=0.05)
    jac = core.schedule_fourier_jacobian(T, n, M)
    phi = synth.random_state(lat.n_qubits, seed=9)

    def value(av):
        psi = core.evolve(lat, c, core.schedule_fourier(T, n, av), T / n, 2)
        if target == "energy":
            return core.energy(psi, lat, c, 1.0)
        return core.fidelity(phi, psi)

    s = core.schedule_fourier(T, n, a)
    if target == "energy":
        v, g = core.energy_gradient(lat, c, s, T / n, 2, jac)
    else:
        v, g = core.fidelity_gradient(lat, c, s, T / n, 2, jac, phi)
    assert v == pytest.approx(value(a), abs=1e-12)
    h = 1e-5
    for m in range(M):
        e = np.zeros(M)
        e[m] = h
        fd = (value(a + e) - value(a - e)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_table1_bound_values():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for n, dg, dt, eps in rows:
        n = int(n)
        dg_, dt_, eps_ = bound.table1_row(n)
        assert dg_ == pytest.approx(float(dg), rel=1e-12)
        assert dt_ == pytest.approx(float(dt), rel=1e-12)
        assert round(eps_, 5) == pytest.approx(float(eps), abs=1e-12)


def test_bound_sum_matches_closed_form():
    p, r, dg, dt = 0.5, 0.05, 1e-3, 2e-2
    a = bound.eps_sum(p, r, dg, dt)
    b = bound.eps_closed(p, r, dg, dt)
    assert a == pytest.approx(b, rel=2e-2)
