"""Warp-local shared passes (QS_OPT_SHARED_KERNEL = 1, k_xpass_wl).

A shared gauge-Higgs pass applies X of one factor group on the pass's new qubits, the
Z layer, and X of the next factor group on the same qubits (Eq. (8): the X-type
factors commute).  When every rotated qubit sits on tile bits 4..11 (a pass fusing at
most 8 new qubits), the tile splits into eight 512-amplitude slices that never
exchange data, and one warp takes a slice through both rounds.  Each amplitude
sees the same floating-point operations in the same order as in the CTA-staged
kernel, so the two agree bit for bit; both match the oracle within the complex64
tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu


def _rel(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return (np.linalg.norm(got - ref) / np.linalg.norm(ref),
            np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def _run(Lx, Ly, plan, kern, nsh, cpl, s, dt, order, psi0=None, renorm=0):
    import torch
    from paper_2108_13410_gb300 import Simulator, QS_OPT_RENORM_EVERY
    from paper_2108_13410_gb300.qsim import (QS_OPT_PLAN, QS_OPT_SHARED_BUFFERS, QS_OPT_SHARED_KERNEL,
                                             plan_code)
    sim = Simulator(Lx, Ly, form="gh", dtype="c64")
    if plan is not None:
        sim.set_option(QS_OPT_PLAN, plan_code(plan))
    sim.set_option(QS_OPT_SHARED_KERNEL, kern)
    sim.set_option(QS_OPT_SHARED_BUFFERS, nsh)
    if renorm:
        sim.set_option(QS_OPT_RENORM_EVERY, renorm)
    if psi0 is None:
        sim.init_plus()
    else:
        sim.upload(torch.from_numpy(psi0.reshape(1, -1)).to(torch.complex64))
    sim.evolve([cpl], s, dt, order)
    return sim.download()[0].numpy()


@gpu
@pytest.mark.parametrize("plan", [[12, 8, 4], [12, 4, 8], [12, 6, 6], [12, 7, 5], [12, 5, 7]])
@pytest.mark.parametrize("order,n_steps", [(2, 3), (1, 2)])
def test_plans_match_the_oracle_and_the_cta_staged_kernel(plan, order, n_steps):
    """2x4 torus, 24 qubits, every pass fusing 4 to 8 new qubits (pass rotations on
    one register layout only, k = 4, or on both): the warp-local shared passes give the
    oracle's amplitudes and the CTA-staged kernel's bits."""
    lat = OracleLattice(2, 4, True, "gh")
    T = 0.2 * n_steps
    s = O.schedule_linear(T, n_steps)
    ref = O.evolve(lat, Couplings(0.7, 0.4), s, T / n_steps, order)
    cta = _run(2, 4, plan, 0, 2, (0.7, 0.4), s, T / n_steps, order)
    for geometry in (0, 2):
        wl = _run(2, 4, plan, 1, geometry, (0.7, 0.4), s, T / n_steps, order)
        rel, mx = _rel(wl, ref)
        assert rel <= 1e-5 and mx <= 1e-5, (geometry, rel, mx)
        assert np.array_equal(wl.view(np.uint32), cta.view(np.uint32)), geometry


@gpu
@pytest.mark.parametrize("nsh", [0, 2, 3])
def test_random_state_fourier_schedule_renormalisation(nsh):
    """3x2 torus (18 qubits: a plain pass and a shared pass fusing 6 new qubits), a
    random complex64 start, a Fourier schedule and renormalisation every 2 steps, in
    the three geometries (one CTA of 24 warps per SM with six tile buffers; three or
    two CTAs of 8 warps with two or three buffers)."""
    lat = OracleLattice(3, 2, True, "gh")
    T, n = 1.0, 7
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(4, seed=11, std=0.05))
    psi0 = synth.random_state(lat.n_qubits, seed=5)
    got = _run(3, 2, None, 1, nsh, (0.9, 0.5), s, T / n, 2, psi0=psi0, renorm=2)
    ref = O.evolve(lat, Couplings(0.9, 0.5), s, T / n, 2, psi0=psi0)
    rel, mx = _rel(got, ref / np.linalg.norm(ref))
    assert rel <= 1e-5 and mx <= 1e-5, (rel, mx)
    cta = _run(3, 2, None, 0, nsh or 2, (0.9, 0.5), s, T / n, 2, psi0=psi0, renorm=2)
    assert np.array_equal(got.view(np.uint32), cta.view(np.uint32))


@gpu
def test_27_qubit_kernels_agree_bit_for_bit_and_match_the_oracle_slice():
    """3x3 torus, 27 qubits (plan 12 + 8 + 7): 12 second-order steps with each shared
    kernel.  The tau = 0 slice equals the 18-qubit unitary-gauge oracle run
    (psi_UG = 2^{9/2} psi_GH(sigma, tau = 0)), and the two kernels agree bit for bit on
    the whole state."""
    import torch
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_SHARED_KERNEL
    ug = OracleLattice(3, 3, True, "ug")
    s = O.schedule_linear(20.0, 1000)[:12]
    ref = O.evolve(ug, Couplings(0.6, 0.6), s, 0.02, 2)
    digests = []
    for kern in (1, 0):
        sim = Simulator(3, 3, form="gh", dtype="c64")
        sim.set_option(QS_OPT_SHARED_KERNEL, kern)
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, 0.02, 2)
        st = sim.state[0]
        if kern == 1:
            sl = st[: 1 << 18].cpu().numpy().astype(np.complex128) * 2 ** 4.5
            rel, mx = _rel(sl, ref)
            assert rel <= 1e-5 and mx <= 1e-5, (rel, mx)
        v = torch.view_as_real(st).view(torch.int32).to(torch.int64)
        w = torch.arange(v.numel(), device=v.device, dtype=torch.int64).view(v.shape) % 65521 + 1
        digests.append(int((v * w).sum().item()))
        del sim, st, v, w
        torch.cuda.empty_cache()
    assert digests[0] == digests[1]


@gpu
def test_option_is_validated():
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300 import qsim as Q
    sim = Simulator(2, 4, form="gh", dtype="c64")
    for bad in (-1, 2):
        with pytest.raises(Q.QsError) as e:
            sim.set_option(Q.QS_OPT_SHARED_KERNEL, bad)
        assert e.value.status == 1


@gpu
@pytest.mark.parametrize("plan", [[12, 8, 4], [12, 4, 8], [12, 6, 6]])
@pytest.mark.parametrize("order,n_steps", [(2, 3), (1, 2)])
def test_unitary_gauge_walsh_hadamard_passes(plan, order, n_steps):
    """3x4 torus in unitary gauge (24 qubits): the shared passes H D_X H and H Z H'
    (Walsh-Hadamard butterflies around the Hadamard-basis X table, with its 2^-24
    scale, or the Z table) on the warp-local kernel give the oracle's amplitudes and the
    CTA-staged kernel's bits."""
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_PLAN, QS_OPT_SHARED_KERNEL, plan_code
    lat = OracleLattice(3, 4, True, "ug")
    T = 0.2 * n_steps
    s = O.schedule_linear(T, n_steps)
    ref = O.evolve(lat, Couplings(0.5, 0.5), s, T / n_steps, order)
    out = []
    for kern in (1, 0):
        sim = Simulator(3, 4, form="ug", dtype="c64")
        sim.set_option(QS_OPT_PLAN, plan_code(plan))
        sim.set_option(QS_OPT_SHARED_KERNEL, kern)
        sim.init_plus()
        sim.evolve([(0.5, 0.5)], s, T / n_steps, order)
        out.append(sim.download()[0].numpy())
    rel, mx = _rel(out[0], ref)
    assert rel <= 1e-5 and mx <= 1e-5, (rel, mx)
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))


@gpu
@pytest.mark.parametrize("T,n", [(2.0, 16), (8.0, 6)])
def test_shared_reverse_passes_match_the_oracle_gradient(T, n):
    """Adjoint on the 3x2 torus (18 qubits; the shared reverse pass fuses 6 qubits) with
    the warp-local shared reverse pass: the gradient of the energy with respect to every
    s_k within the complex64 tolerance (1e-3 of the largest oracle component), the value
    within 1e-4 relative, psi uncomputed back to |+>; the CTA-staged reverse pass gives
    the same value bit for bit (same forward) and the gradient up to float summation
    order.  T = 2, 16 steps runs the tangent form (shared reverse passes); T = 8, 6 steps
    (X angles near 1) the (u, s) rotations without shared reverse passes."""
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_SHARED_KERNEL
    lat = OracleLattice(3, 2, True, "gh")
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(4, seed=7, std=0.05))
    e_ref, g_ref = O.energy_gradient(lat, Couplings(0.6, 0.6), s, T / n, 2, np.eye(n))
    res = []
    for kern in (1, 0):
        sim = Simulator(3, 2, form="gh", dtype="c64", aux=True)
        sim.set_option(QS_OPT_SHARED_KERNEL, kern)
        sim.init_plus()
        val, g = sim.adjoint_grad([(0.6, 0.6)], s, T / n, 2)
        res.append((val[0], g[0]))
        if kern == 1:
            assert abs(val[0] - e_ref) <= 1e-4 * abs(e_ref)
            scale = np.max(np.abs(g_ref))
            assert np.max(np.abs(g[0] - g_ref)) <= 1e-3 * scale
            psi0 = sim.download()[0].numpy().astype(np.complex128)
            assert np.linalg.norm(psi0 - O.plus_state(lat.n_qubits)) <= 1e-4
    assert res[0][0] == res[1][0]
    assert np.max(np.abs(res[0][1] - res[1][1])) <= 1e-5 * np.max(np.abs(res[1][1]))


@gpu
def test_27_qubit_shared_reverse_passes_agree():
    """3x3 torus, 27 qubits, 40 steps of the Fourier schedule: the warp-local and the
    CTA-staged shared reverse passes give the same value (same forward) and gradients
    within 1e-5 of the largest component (float summation order of the terms)."""
    import torch
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_SHARED_KERNEL
    T, n = 1.6, 40
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(8, seed=3, std=0.02))
    res = []
    for kern in (1, 0):
        sim = Simulator(3, 3, form="gh", dtype="c64", aux=True)
        sim.set_option(QS_OPT_SHARED_KERNEL, kern)
        sim.init_plus()
        val, g = sim.adjoint_grad([(0.6, 0.6)], s, T / n, 2)
        res.append((val[0], g[0]))
        del sim
        torch.cuda.empty_cache()
    assert res[0][0] == res[1][0]
    assert np.max(np.abs(res[0][1] - res[1][1])) <= 1e-5 * np.max(np.abs(res[1][1]))


@gpu
@pytest.mark.parametrize("lattice,form", [((2, 2), "gh"), ((3, 2), "ug"), ((4, 2), "ug")],
                         ids=["gh2x2open-21q", "ug3x2open-17q", "ug4x2open-22q"])
def test_open_lattices_edge_passes(lattice, form):
    """Open lattices whose shared passes are edge cases of the slice split: 21 qubits
    (gauge-Higgs, plan 12 + 8 + 1: a pass rotating tile bit 11 alone), 17 qubits (unitary
    gauge, 12 + 5: 32 tiles for 152 CTAs, most of which get no tile) and 22 qubits
    (unitary gauge, 12 + 8 + 2).  Oracle parity and bit-identity with the CTA-staged
    kernel."""
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_SHARED_KERNEL
    Lx, Ly = lattice
    lat = OracleLattice(Lx, Ly, False, form)
    n_steps = 3
    T = 0.15 * n_steps
    s = O.schedule_linear(T, n_steps)
    ref = O.evolve(lat, Couplings(0.7, 0.4), s, T / n_steps, 2)
    out = []
    for kern in (1, 0):
        sim = Simulator(Lx, Ly, form=form, dtype="c64", boundary="open")
        sim.set_option(QS_OPT_SHARED_KERNEL, kern)
        sim.init_plus()
        sim.evolve([(0.7, 0.4)], s, T / n_steps, 2)
        out.append(sim.download()[0].numpy())
    rel, mx = _rel(out[0], ref)
    assert rel <= 1e-5 and mx <= 1e-5, (rel, mx)
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))
