"""Pin of where the schedule is sampled within a Trotter step.

Sec. III carries the ground state along the path by steps of equal duration, each
step a product formula (Eq. (7)) of H at one value of the schedule.  The reading
used here samples s at the step midpoints, t_k = (k - 1/2) dt.  Against the exact
time-ordered evolution of the continuous ramp, T exp(-i int_0^T H(s(t)) dt), the
second-order product then keeps a global error of order dt^2; sampling at the step
ends instead (a plausible mistake) makes the discretisation of time first order,
whatever the order of the product.

The continuous evolution is integrated with the fourth-order Magnus method (two
Gauss-Legendre points per sub-step), on dense matrices of H(s) on the 2x2 torus in
the unitary gauge (256 states), with enough sub-steps that its own error is far
below the Trotter errors measured.
"""
import math

import numpy as np

from oracle import OracleLattice, Couplings
from oracle import core, ed

T = 2.0
C = Couplings(0.6, 0.6)


def _continuous_reference(lat, s_of_t, substeps):
    """T exp(-i int H(s(t)) dt) |+>, fourth-order Magnus: per sub-step of length h,
    Omega = -i h (H1 + H2)/2 + (sqrt(3) h^2 / 12) [H1, H2] with H1, H2 at the Gauss
    points t0 + h (1/2 -+ sqrt(3)/6)."""
    psi = core.plus_state(lat.n_qubits)
    h = T / substeps
    c1, c2 = 0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6
    # H(s) = (1 - s) H0 + s H1 is affine in s
    H_0 = ed.dense(ed.hamiltonian(lat, C, 0.0))
    H_1 = ed.dense(ed.hamiltonian(lat, C, 1.0))
    H = lambda s: H_0 + s * (H_1 - H_0)
    for k in range(substeps):
        t0 = k * h
        H1 = H(s_of_t(t0 + c1 * h))
        H2 = H(s_of_t(t0 + c2 * h))
        # Omega = -i K with K = h (H1 + H2)/2 + i (sqrt(3) h^2 / 12) [H1, H2] Hermitian
        K = 0.5 * h * (H1 + H2) + 1j * (math.sqrt(3) * h * h / 12.0) * (H1 @ H2 - H2 @ H1)
        w, V = np.linalg.eigh(K)
        psi = V @ (np.exp(-1j * w) * (V.conj().T @ psi))
    return psi


def _slope(errs, steps):
    return -np.polyfit(np.log(steps), np.log(errs), 1)[0]


def test_midpoint_sampling_gives_second_order_against_continuous_ramp():
    lat = OracleLattice(2, 2, True, "ug")
    ramp = lambda t: t / T
    ref = _continuous_reference(lat, ramp, 120)
    ref_fine = _continuous_reference(lat, ramp, 240)
    assert np.linalg.norm(ref - ref_fine) < 1e-7          # the reference is converged
    steps = np.array([10, 20, 40, 80])
    mid, ends = [], []
    for n in steps:
        dt = T / n
        s_mid = core.schedule_linear(T, n)                  # the oracle's sampling
        s_end = np.arange(1, n + 1) * dt / T                # sampled at the step ends
        assert np.allclose(s_mid, (np.arange(1, n + 1) - 0.5) * dt / T)
        mid.append(np.linalg.norm(core.evolve(lat, C, s_mid, dt, 2) - ref))
        ends.append(np.linalg.norm(core.evolve(lat, C, s_end, dt, 2) - ref))
    assert abs(_slope(mid, steps) - 2.0) <= 0.15, mid
    assert _slope(ends, steps) <= 1.3, ends
    assert all(m < e for m, e in zip(mid[1:], ends[1:]))
    # first order: the product formula itself limits the slope to 1 either way
    first = [np.linalg.norm(core.evolve(lat, C, core.schedule_linear(T, n), T / n, 1) - ref) for n in steps]
    assert abs(_slope(first, steps) - 1.0) <= 0.15, first
