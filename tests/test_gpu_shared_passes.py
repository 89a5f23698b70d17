"""Shared passes (QS_OPT_XMERGE): consecutive Trotter factor groups take their qubit
groups in opposite orders, and the pass of the group they meet on applies X of one
factor group, the Z layer, and X of the next (all X-type factors commute, Eq. (8)).

The operator sequence is unchanged, so the amplitudes equal the oracle's within the
complex64 tolerance (||d psi|| / ||psi|| <= 1e-5, and the same bound on the largest
amplitude error relative to the largest amplitude).
"""
import numpy as np
import pytest

import synth
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
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("n_steps", [1, 2, 5, 16])
@pytest.mark.parametrize("store", [0, 1])
def test_two_pass_lattice_matches_oracle(order, n_steps, store):
    """3x2 torus, gauge-Higgs form: 18 qubits, two passes per X layer, so every
    factor group after the first costs one pass.  Batch 2 with different couplings."""
    from paper_2108_13410_gb300.qsim import QS_OPT_TMA_STORE
    lat = OracleLattice(3, 2, True, "gh")
    couplings = [(0.6, 0.6), (1.1, 0.3)]
    T = 0.2 * n_steps
    s = O.schedule_linear(T, n_steps)
    sim = _sim(3, 2, form="gh", dtype="c64", batch=2)
    sim.set_option(QS_OPT_TMA_STORE, store)
    sim.init_plus()
    sim.evolve(couplings, s, T / n_steps, order)
    got = sim.download().numpy()
    for b, (g, lam) in enumerate(couplings):
        _assert_amplitudes(got[b], O.evolve(lat, Couplings(g, lam), s, T / n_steps, order))


@gpu
@pytest.mark.parametrize("order,n_steps", [(2, 1), (2, 4), (1, 3)])
@pytest.mark.parametrize("nsh", [2, 3])
def test_three_pass_lattice_matches_oracle(order, n_steps, nsh):
    """2x4 torus, gauge-Higgs form: 24 qubits, three passes per X layer (qubits
    0-11, 12-19, 20-23): the shared pass alternates between the second and the third
    qubit group, the first runs alone in the middle of every factor group.  Shared
    passes with 2 or 3 tile buffers (QS_OPT_SHARED_BUFFERS)."""
    from paper_2108_13410_gb300.qsim import QS_OPT_SHARED_BUFFERS
    lat = OracleLattice(2, 4, True, "gh")
    c = Couplings(0.7, 0.4)
    T = 0.15 * n_steps
    s = O.schedule_linear(T, n_steps)
    sim = _sim(2, 4, form="gh", dtype="c64")
    sim.set_option(QS_OPT_SHARED_BUFFERS, nsh)
    sim.init_plus()
    sim.evolve([(0.7, 0.4)], s, T / n_steps, order)
    _assert_amplitudes(sim.download()[0].numpy(), O.evolve(lat, c, s, T / n_steps, order))


@gpu
def test_shared_passes_from_a_random_state_with_renormalisation():
    """Random complex64 start (every amplitude and phase exercised), renormalisation
    every 2 steps between shared passes, Fourier schedule."""
    from paper_2108_13410_gb300 import QS_OPT_RENORM_EVERY
    import torch
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(0.9, 0.5)
    T, n = 1.0, 7
    a = synth.fourier_coeffs(4, seed=11, std=0.05)
    s = O.schedule_fourier(T, n, a)
    psi0 = synth.random_state(lat.n_qubits, seed=5)
    sim = _sim(3, 2, form="gh", dtype="c64")
    sim.set_option(QS_OPT_RENORM_EVERY, 2)
    sim.upload(torch.from_numpy(psi0.reshape(1, -1)).to(torch.complex64))
    sim.evolve([(0.9, 0.5)], s, T / n, 2)
    ref = O.evolve(lat, c, s, T / n, 2, psi0=psi0)
    _assert_amplitudes(sim.download()[0].numpy(), ref / np.linalg.norm(ref))


@gpu
def test_shared_and_separate_passes_agree_across_a_record_chunk():
    """A gauge-Higgs path of 2050 steps (more than the 2048 factor groups whose records
    are resident at once): the shared-pass chain restarts at the chunk boundary.  A
    dropped or repeated factor would change the state by O(dt); the two schedules
    differ only in rounding order."""
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    path = [(0.2 + 1e-4 * k, 0.5 - 1e-4 * k, 1.0, 1.0) for k in range(2050)]
    out = []
    for merge in (1, 0):
        sim = _sim(3, 2, form="gh", dtype="c64")
        sim.set_option(QS_OPT_XMERGE, merge)
        sim.init_plus()
        sim.evolve_path(path, 0.02, 2)
        out.append(sim.download()[0].numpy().astype(np.complex128))
    assert np.linalg.norm(out[0] - out[1]) <= 1e-4


@gpu
def test_shared_passes_at_27_qubits_agree_with_separate_passes():
    """3x3 torus (27 qubits, three passes per X layer): 20 second-order steps with and
    without shared passes, both in complex64, agree within the complex64 tolerance;
    sampled amplitudes and the energy."""
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    import torch
    s = O.schedule_linear(20.0, 1000)[:20]
    idx = torch.from_numpy(np.random.default_rng(3).integers(0, 1 << 27, 4096))
    amps, es = [], []
    for merge in (1, 0):
        sim = _sim(3, 3, form="gh", dtype="c64")
        sim.set_option(QS_OPT_XMERGE, merge)
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, 0.02, 2)
        amps.append(sim.state[0, idx.to(sim.state.device)].cpu().numpy().astype(np.complex128))
        es.append(sim.energy([(0.6, 0.6)])[0])
        del sim
        torch.cuda.empty_cache()
    scale = np.max(np.abs(amps[1]))
    assert np.max(np.abs(amps[0] - amps[1])) <= 1e-5 * scale
    assert abs(es[0] - es[1]) <= 1e-4


@gpu
@pytest.mark.parametrize("order,n_steps", [(1, 1), (2, 1), (2, 3), (1, 4)])
@pytest.mark.parametrize("store", [0, 1])
def test_unitary_gauge_shared_passes_match_oracle(order, n_steps, store):
    """3x3 torus, unitary gauge (18 link qubits, two passes per Walsh-Hadamard round):
    a factor group is [H(q0-11) Z H(q0-11)] and [H(q12-17) D_X H(q12-17)], two passes
    instead of four."""
    from paper_2108_13410_gb300.qsim import QS_OPT_TMA_STORE
    lat = OracleLattice(3, 3, True, "ug")
    c = Couplings(0.3, 0.5, J=0.5, h=0.5)
    T = 0.2 * n_steps
    s = O.schedule_linear(T, n_steps)
    sim = _sim(3, 3, form="ug", dtype="c64")
    sim.set_option(QS_OPT_TMA_STORE, store)
    sim.init_plus()
    sim.evolve([(0.3, 0.5, 0.5, 0.5)], s, T / n_steps, order)
    _assert_amplitudes(sim.download()[0].numpy(), O.evolve(lat, c, s, T / n_steps, order))


@gpu
def test_unitary_gauge_shared_passes_batch_and_toric_start():
    """2x5 torus, unitary gauge (20 qubits), batch 2, from the toric-code state psi_1
    along two different parameter paths."""
    lat = OracleLattice(2, 5, True, "ug")
    paths = [[(0.01 * k, 0.3, 0.5, 0.5) for k in range(1, 7)], [(0.2, 0.02 * k, 0.5, 0.5) for k in range(1, 7)]]
    sim = _sim(2, 5, form="ug", dtype="c64", batch=2)
    sim.init_toric(0)
    per_step = [[paths[0][k], paths[1][k]] for k in range(6)]
    sim.evolve_path(per_step, 0.05, 2)
    got = sim.download().numpy()
    psi0 = O.toric_state(lat, 0)
    for b in range(2):
        ref = O.evolve_path(lat, [Couplings(g, l, J=J, h=h) for g, l, J, h in paths[b]], 0.05, 2, psi0=psi0)
        _assert_amplitudes(got[b], ref)


@gpu
def test_unitary_gauge_launch_count():
    """Unitary gauge 3x3 (two passes per Walsh-Hadamard round): 10 second-order steps =
    11 factor groups; shared passes: 1 + 2 per group; separate: 4 per group."""
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    sim = _sim(3, 3, form="ug", dtype="c64")
    sim.init_plus()
    sim.launch_count()
    s = O.schedule_linear(1.0, 10)
    sim.evolve([(0.6, 0.6)], s, 0.1, 2)
    sim.sync()
    assert sim.launch_count() == 1 + 1 + 2 * 11      # records + first H pass + 2 per group
    sim.set_option(QS_OPT_XMERGE, 0)
    sim.evolve([(0.6, 0.6)], s, 0.1, 2)
    sim.sync()
    assert sim.launch_count() == 1 + 4 * 11


@gpu
def test_unitary_gauge_32_qubits_shared_and_separate_passes_agree():
    """4x4 torus, unitary gauge (32 qubits, four passes per Walsh-Hadamard round: six
    instead of eight per factor group): three second-order steps with and without
    shared passes agree on sampled amplitudes."""
    import torch
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    s = [0.2, 0.4, 0.6]
    idx = torch.from_numpy(np.random.default_rng(6).integers(0, 1 << 32, 4096))
    amps = []
    for merge in (1, 0):
        sim = _sim(4, 4, form="ug", dtype="c64")
        sim.set_option(QS_OPT_XMERGE, merge)
        sim.init_plus()
        sim.evolve([(0.5, 0.5)], s, 0.1, 2)
        amps.append(sim.state[0, idx.to(sim.state.device)].cpu().numpy().astype(np.complex128))
        del sim
        torch.cuda.empty_cache()
    scale = np.max(np.abs(amps[1]))
    assert np.max(np.abs(amps[0] - amps[1])) <= 1e-5 * scale
