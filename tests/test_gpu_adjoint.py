"""Adjoint gradient (qs_adjoint_grad) against the oracle's forward-mode tangents and
against central finite differences of the GPU evolution.

Tolerances: complex128 gradients agree with the FP64 oracle to 1e-8 relative to the
largest component; complex64 to 1e-3 relative (the complex64 amplitudes carry ~1e-6
relative error, and each dV/ds_k sums many products of them).
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


def _close(got, ref, rel):
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= rel * scale + 1e-12, (np.max(np.abs(got - ref)), scale)


def _tol(dtype):
    return 1e-8 if dtype == "c128" else 1e-3


@gpu
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("lattice", [(2, 2), (3, 2)])
def test_energy_gradient_matches_oracle(dtype, order, lattice):
    Lx, Ly = lattice
    lat = OracleLattice(Lx, Ly, True, "gh")
    c = Couplings(0.6, 0.6)
    T, n = 2.0, 16
    a = synth.fourier_coeffs(4, seed=7, std=0.05)
    s = O.schedule_fourier(T, n, a)
    # dE/ds_k for every k: tangents seeded with the identity
    e_ref, g_ref = O.energy_gradient(lat, c, s, T / n, order, np.eye(n))
    sim = _sim(Lx, Ly, form="gh", dtype=dtype, aux=True)
    sim.init_plus()
    val, g = sim.adjoint_grad([(0.6, 0.6)], s, T / n, order)
    assert abs(val[0] - e_ref) <= (1e-9 if dtype == "c128" else 1e-4 * abs(e_ref))
    _close(g[0], g_ref, _tol(dtype))
    # psi is uncomputed back to |+>
    psi0 = sim.download()[0].numpy().astype(np.complex128)
    drift = np.linalg.norm(psi0 - O.plus_state(lat.n_qubits))
    assert drift <= (1e-11 if dtype == "c128" else 1e-4)


@gpu
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fidelity_gradient_matches_oracle(dtype):
    import torch
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(0.9, 0.4)
    T, n, M = 2.0, 12, 3
    a = synth.fourier_coeffs(M, seed=8, std=0.05)
    s = O.schedule_fourier(T, n, a)
    jac = O.schedule_fourier_jacobian(T, n, M)
    phi = synth.random_state(lat.n_qubits, seed=31)
    f_ref, gf_ref = O.fidelity_gradient(lat, c, s, T / n, 2, jac, phi)
    sim = _sim(3, 2, form="gh", dtype=dtype, aux=True)
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    phi_dev = torch.from_numpy(phi.reshape(1, -1)).to(tdt).cuda()
    sim.init_plus()
    val, g = sim.adjoint_grad([(0.9, 0.4)], s, T / n, 2, target="fidelity", ref_state=phi_dev)
    assert abs(val[0] - f_ref) <= (1e-12 if dtype == "c128" else 1e-6)
    _close(jac @ g[0], gf_ref, _tol(dtype))


@gpu
def test_batched_adjoint_is_per_element():
    couplings = [(0.2, 0.2), (0.6, 0.6)]
    T, n = 2.0, 10
    s = O.schedule_linear(T, n)
    sim = _sim(2, 2, form="gh", dtype="c128", batch=2, aux=True)
    sim.init_plus()
    val, g = sim.adjoint_grad(couplings, s, T / n, 2)
    lat = OracleLattice(2, 2, True, "gh")
    for b, (gg, lam) in enumerate(couplings):
        e_ref, g_ref = O.energy_gradient(lat, Couplings(gg, lam), s, T / n, 2, np.eye(n))
        assert abs(val[b] - e_ref) <= 1e-9
        _close(g[b], g_ref, 1e-8)


@gpu
def test_adjoint_matches_finite_differences_on_the_gpu_path():
    """Central differences (h = 1e-4) of the complex128 GPU energy in the Fourier
    amplitudes a_m against the adjoint chained through the autograd Function."""
    import torch
    from paper_2108_13410_gb300.autograd import schedule_value, fourier_schedule
    T, n, M = 2.0, 20, 4
    a0 = synth.fourier_coeffs(M, seed=2108, std=0.01)
    sim = _sim(3, 2, form="gh", dtype="c128", aux=True)
    cpl = [(0.6, 0.6)]
    a = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    e = schedule_value(a, sim, cpl, T, n)
    e.backward()

    def energy(av):
        s, _ = fourier_schedule(av, T, n)
        sim.init_plus()
        sim.evolve(cpl, s, T / n, 2)
        return sim.energy(cpl)[0]

    h = 1e-4
    fd = []
    for m in range(M):
        d = np.zeros(M)
        d[m] = h
        fd.append((energy(a0 + d) - energy(a0 - d)) / (2 * h))
    fd = np.array(fd)
    assert np.max(np.abs(a.grad.numpy() - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd)))


@gpu
@pytest.mark.parametrize("L", [(2, 2), (3, 2)])
def test_batched_complex64_adjoint_tma_path(L):
    """complex64 adjoint (TMA reverse pass) with two batch elements: per-element sums."""
    couplings = [(0.2, 0.9), (0.6, 0.6)]
    T, n = 2.0, 12
    s = O.schedule_linear(T, n)
    sim = _sim(*L, form="gh", dtype="c64", batch=2, aux=True)
    sim.init_plus()
    val, g = sim.adjoint_grad(couplings, s, T / n, 2)
    lat = OracleLattice(*L, True, "gh")
    for b, (gg, lam) in enumerate(couplings):
        e_ref, g_ref = O.energy_gradient(lat, Couplings(gg, lam), s, T / n, 2, np.eye(n))
        assert abs(val[b] - e_ref) <= 1e-4 * abs(e_ref)
        _close(g[b], g_ref, 1e-3)
    psi0 = sim.download().numpy().astype(np.complex128)
    for b in range(2):
        assert np.linalg.norm(psi0[b] - O.plus_state(lat.n_qubits)) <= 1e-4


@gpu
@pytest.mark.parametrize("T,n", [(2.0, 16), (8.0, 8)])
@pytest.mark.parametrize("adj", [0, 2, 4])
@pytest.mark.parametrize("merge", [1, 0])
def test_complex64_adjoint_forms_and_buffers(T, n, adj, merge):
    """complex64 adjoint on the 3x2 torus in both forms of the reverse pass: small angles
    (T = 2, 16 steps) run the tangent form, large angles (T = 8, 8 steps: X angles
    near 1) the (u, s) rotations; one tile-pair buffer with the next load issued before
    the per-thread stores (QS_OPT_ADJOINT 0), two buffers (2), one buffer with bulk
    tensor stores (4).
    Gradient within 1e-3 of the largest oracle component, value within 1e-4 relative,
    psi uncomputed back to |+> within 1e-4.  With shared passes (QS_OPT_XMERGE 1) the
    tangent-form reverse sweep shares one pass between consecutive factor groups."""
    from paper_2108_13410_gb300.qsim import QS_OPT_ADJOINT, QS_OPT_XMERGE
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(0.6, 0.6)
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(4, seed=7, std=0.05))
    e_ref, g_ref = O.energy_gradient(lat, c, s, T / n, 2, np.eye(n))
    sim = _sim(3, 2, form="gh", dtype="c64", aux=True)
    sim.set_option(QS_OPT_ADJOINT, adj)
    sim.set_option(QS_OPT_XMERGE, merge)
    for _ in range(2):                       # twice in a row: nothing left over between calls
        sim.init_plus()
        val, g = sim.adjoint_grad([(0.6, 0.6)], s, T / n, 2)
        assert abs(val[0] - e_ref) <= 1e-4 * abs(e_ref)
        _close(g[0], g_ref, 1e-3)
        psi0 = sim.download()[0].numpy().astype(np.complex128)
        assert np.linalg.norm(psi0 - O.plus_state(lat.n_qubits)) <= 1e-4


@gpu
def test_shared_reverse_passes_across_a_record_chunk():
    """3x2 torus (18 qubits, two passes per X layer), 2100 second-order steps (more than
    the 2048 factor groups whose records are resident at once): the adjoint with shared
    reverse passes gives the gradient of the adjoint with separate passes within 1e-3 of
    its largest component, the complex64 tolerance (measured: 1.1e-4, rounding accumulated
    over 2100 steps; a factor dropped or repeated at the chunk boundary, where the chain of
    shared passes restarts, would differ by the size of the gradient), and the same value."""
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    T, n = 42.0, 2100
    s = O.schedule_linear(T, n)
    res = []
    for merge in (1, 0):
        sim = _sim(3, 2, form="gh", dtype="c64", aux=True)
        sim.set_option(QS_OPT_XMERGE, merge)
        sim.init_plus()
        res.append(sim.adjoint_grad([(0.6, 0.6)], s, T / n, 2))
    (v1, g1), (v0, g0) = res
    assert abs(v1[0] - v0[0]) <= 1e-4 * abs(v0[0])
    _close(g1[0], g0[0], 1e-3)
