"""Tangent form of the complex64 X passes: in the real-rotation frame each factor
exp(i theta X) is cos theta [[1, t], [-t, 1]], t = tan theta, and the cos factors of
a factor group are applied once as a scalar C, carried by the Z table (each entry's
modulus chosen to be C).  Used when every factor group of a call has |theta| <= pi/4
and C >= 1/2; otherwise the (u, s) form runs.  Tolerances as in the parity tests
(complex64: 1e-5 relative)."""
import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu


def _sim(*a, **k):
    from paper_2108_13410_gb300 import Simulator
    return Simulator(*a, **k)


def _assert_amplitudes(got, ref, tol=1e-5):
    got = np.asarray(got, dtype=np.complex128)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert rel <= tol and mx <= tol, (rel, mx, tol)


@gpu
@pytest.mark.parametrize("dt", [0.05, 0.3, 1.3])
def test_angles_across_the_forms(dt):
    """s = 0.2, X coefficients 1.04 and 1.0 on 18 qubits: at dt = 0.05 the tangent
    form runs (C ~ 0.99); at dt = 0.3 the first-order step has C < 1/2 and runs the
    (u, s) rotations while the second-order step (half angles, C ~ 0.8) runs the
    tangent form; at dt = 1.3 the angles exceed pi/4.  All equal the oracle's step."""
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(1.2, 0.4)
    sim = _sim(3, 2, form="gh", dtype="c64")
    for order in (1, 2):
        sim.init_plus()
        sim.trotter_step([(1.2, 0.4)], 0.2, dt, order)
        ref = O.plus_state(lat.n_qubits)
        O.trotter_step(ref, lat, c, 0.2, dt, order)
        _assert_amplitudes(sim.download()[0].numpy(), ref)


@gpu
def test_angles_at_the_switch_point():
    """First order at s = 0 (theta = dt for all 18 X qubits, no Z angles): C = (1 +
    tan^2 dt)^(-9) crosses 1/2 at tan dt = (4^(1/9) - 1)^(1/2); one call just below and
    one just above."""
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(0.6, 0.6)
    sim = _sim(3, 2, form="gh", dtype="c64")
    th = np.arctan(np.sqrt(4.0 ** (1.0 / 9.0) - 1.0))
    for dt in (th - 1e-3, th + 1e-3):
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], [0.0, 0.0], dt, 1)
        ref = O.evolve(lat, c, [0.0, 0.0], dt, 1)
        _assert_amplitudes(sim.download()[0].numpy(), ref)


@gpu
def test_norm_is_kept_over_a_long_run():
    """1500 second-order steps without renormalisation: with C carried by the scaled Z
    table (modulus C to ~1e-10 per entry) |norm - 1| stays far below the up to ~3e-8
    per factor group (up to 4.5e-5 after 1500 groups) that rounding C to a float would
    leave."""
    from paper_2108_13410_gb300 import QS_NORM
    sim = _sim(3, 2, form="gh", dtype="c64")
    sim.init_plus()
    s = O.schedule_linear(30.0, 1500)
    sim.evolve([(0.6, 0.6)], s, 0.02, 2)
    assert abs(sim.expect(QS_NORM)[0] - 1.0) <= 1e-6


@gpu
def test_tangent_and_rotation_forms_agree_at_27_qubits():
    """The same 30 steps at 27 qubits with the tangent form (default) and with the
    rotation form (forced by a call whose first angle is large, then the same steps):
    sampled amplitudes agree within the complex64 tolerance."""
    import torch
    from paper_2108_13410_gb300.qsim import QS_OPT_XPASS
    s = O.schedule_linear(20.0, 1000)[:30]
    idx = torch.from_numpy(np.random.default_rng(4).integers(0, 1 << 27, 4096))
    amps = []
    for impl in (0, 1):          # TMA kernel (tangent form) / register kernel ((u, s) form)
        sim = _sim(3, 3, form="gh", dtype="c64")
        sim.set_option(QS_OPT_XPASS, impl)
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, 0.02, 2)
        amps.append(sim.state[0, idx.to(sim.state.device)].cpu().numpy().astype(np.complex128))
        del sim
        torch.cuda.empty_cache()
    scale = np.max(np.abs(amps[1]))
    assert np.max(np.abs(amps[0] - amps[1])) <= 1e-5 * scale
