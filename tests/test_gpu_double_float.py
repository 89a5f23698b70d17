"""complex128 unitary-gauge passes in double-float arithmetic (QS_OPT_C128_DF, default on).

Each real number is an unevaluated sum of two floats (48 significand bits); sums and
differences use two-sum with renormalisation, products the exact FMA high product.  A
pass keeps the FP64 oracle's amplitudes to the complex128 tolerance (1e-10 of the norm and
of the largest amplitude), and agrees with the FP64 register kernel to ~1e-13.
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


def _run(Lx, Ly, df, couplings, s, dt, order, batch=1, psi0=None, renorm=0, plan=None):
    import torch
    from paper_2108_13410_gb300 import Simulator, QS_OPT_RENORM_EVERY
    from paper_2108_13410_gb300.qsim import QS_OPT_C128_DF, QS_OPT_PLAN, plan_code
    sim = Simulator(Lx, Ly, form="ug", dtype="c128", batch=batch)
    sim.set_option(QS_OPT_C128_DF, df)
    if plan is not None:
        sim.set_option(QS_OPT_PLAN, plan_code(plan))
    if renorm:
        sim.set_option(QS_OPT_RENORM_EVERY, renorm)
    if psi0 is None:
        sim.init_plus()
    else:
        sim.upload(torch.from_numpy(np.tile(psi0, (batch, 1))))
    sim.evolve(couplings, s, dt, order)
    return sim.download().numpy()


@gpu
@pytest.mark.parametrize("order,n_steps", [(2, 3), (1, 2)])
@pytest.mark.parametrize("plan", [None, [12, 4, 8], [12, 6, 6]])
def test_24_qubit_unitary_gauge_matches_oracle(order, n_steps, plan):
    """3x4 torus in unitary gauge (24 qubits, three passes per transform, shared passes
    H D_X H and H Z H'): double-float passes against the FP64 oracle at 1e-10, and against
    the FP64 register kernel."""
    lat = OracleLattice(3, 4, True, "ug")
    T = 0.3 * n_steps
    s = O.schedule_linear(T, n_steps)
    ref = O.evolve(lat, Couplings(0.5, 0.5), s, T / n_steps, order)
    df = _run(3, 4, 1, [(0.5, 0.5)], s, T / n_steps, order, plan=plan)[0]
    rel, mx = _rel(df, ref)
    assert rel <= 1e-10 and mx <= 1e-10, (rel, mx)
    fp64 = _run(3, 4, 0, [(0.5, 0.5)], s, T / n_steps, order, plan=plan)[0]
    rel, mx = _rel(df, fp64)
    assert rel <= 1e-12 and mx <= 1e-12, (rel, mx)


@gpu
def test_random_state_batch_and_renormalisation():
    """3x3 unitary gauge (18 qubits, two passes), batch 2 with different couplings, a
    random complex128 start, a Fourier schedule and renormalisation every 2 steps (the
    state is joined to complex128 for the rescale and split again)."""
    lat = OracleLattice(3, 3, True, "ug")
    T, n = 1.2, 6
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(4, seed=13, std=0.05))
    psi0 = synth.random_state(lat.n_qubits, seed=9).astype(np.complex128)
    cps = [(0.7, 0.3), (0.2, 1.1)]
    got = _run(3, 3, 1, cps, s, T / n, 2, batch=2, psi0=psi0, renorm=2)
    for b, (g, lam) in enumerate(cps):
        ref = O.evolve(lat, Couplings(g, lam), s, T / n, 2, psi0=psi0)
        rel, mx = _rel(got[b], ref / np.linalg.norm(ref))
        assert rel <= 1e-10 and mx <= 1e-10, (b, rel, mx)


@gpu
def test_identity_step_round_trip():
    """One step with dt = 0 (every factor the identity): split into the blocked layout,
    unnormalised transforms there and back with the identity table between them and the
    2^-18 scale, join.  A random state comes back to double-float rounding of the 36
    butterfly stages (1e-12 of its largest amplitude)."""
    import torch
    from paper_2108_13410_gb300 import Simulator
    sim = Simulator(3, 3, form="ug", dtype="c128")
    psi0 = synth.random_state(18, seed=4).astype(np.complex128)
    sim.upload(torch.from_numpy(psi0.reshape(1, -1)))
    sim.evolve([(0.5, 0.5)], [0.5], 0.0, 2)     # dt = 0: identity factors around split / join
    got = sim.download().numpy()[0]
    assert np.max(np.abs(got - psi0)) <= 1e-12 * np.max(np.abs(psi0))


def _run_gh(Lx, Ly, df, couplings, s, dt, order, batch=1, xmerge=1, renorm=0, psi0=None):
    import torch
    from paper_2108_13410_gb300 import Simulator, QS_OPT_RENORM_EVERY
    from paper_2108_13410_gb300.qsim import QS_OPT_C128_DF, QS_OPT_XMERGE
    sim = Simulator(Lx, Ly, form="gh", dtype="c128", batch=batch)
    sim.set_option(QS_OPT_C128_DF, df)
    sim.set_option(QS_OPT_XMERGE, xmerge)
    if renorm:
        sim.set_option(QS_OPT_RENORM_EVERY, renorm)
    if psi0 is None:
        sim.init_plus()
    else:
        sim.upload(torch.from_numpy(np.tile(psi0, (batch, 1))))
    sim.evolve(couplings, s, dt, order)
    return sim.download().numpy()


@gpu
@pytest.mark.parametrize("lattice,order,n_steps,xmerge",
                         [((3, 2), 2, 6, 1), ((3, 2), 1, 4, 1), ((2, 4), 2, 3, 1), ((2, 4), 1, 3, 0)])
def test_gauge_higgs_tangent_form_matches_oracle(lattice, order, n_steps, xmerge):
    """Gauge-Higgs form in complex128 with double-float passes (tangent-form rotations in
    the real frame, the C-scaled Z table, shared passes or separate ones): batch 2 on the
    3x2 torus (18 qubits, two passes) and one state on the 2x4 torus (24 qubits, three
    passes) against the FP64 oracle at 1e-10 and the FP64 register kernel at 1e-12."""
    Lx, Ly = lattice
    lat = OracleLattice(Lx, Ly, True, "gh")
    T = 0.15 * n_steps
    s = O.schedule_linear(T, n_steps)
    cps = [(0.6, 0.6), (1.1, 0.3)] if lattice == (3, 2) else [(0.7, 0.4)]
    got = _run_gh(Lx, Ly, 1, cps, s, T / n_steps, order, batch=len(cps), xmerge=xmerge)
    fp64 = _run_gh(Lx, Ly, 0, cps, s, T / n_steps, order, batch=len(cps), xmerge=xmerge)
    for b, (g, lam) in enumerate(cps):
        ref = O.evolve(lat, Couplings(g, lam), s, T / n_steps, order)
        rel, mx = _rel(got[b], ref)
        assert rel <= 1e-10 and mx <= 1e-10, (b, rel, mx)
        rel, mx = _rel(got[b], fp64[b])
        assert rel <= 1e-12 and mx <= 1e-12, (b, rel, mx)


@gpu
def test_gauge_higgs_large_angles_and_renormalisation():
    """Large X angles (dt = 0.9: outside the tangent form's range) run the FP64 kernel
    and still match the oracle; a random start with renormalisation every 2 steps runs
    the double-float passes (joined for each rescale)."""
    lat = OracleLattice(3, 2, True, "gh")
    s = O.schedule_linear(1.8, 2)
    got = _run_gh(3, 2, 1, [(0.6, 0.6)], s, 0.9, 2)[0]
    rel, mx = _rel(got, O.evolve(lat, Couplings(0.6, 0.6), s, 0.9, 2))
    assert rel <= 1e-10 and mx <= 1e-10, (rel, mx)
    T, n = 1.0, 7
    s = O.schedule_fourier(T, n, synth.fourier_coeffs(4, seed=11, std=0.05))
    psi0 = synth.random_state(lat.n_qubits, seed=5).astype(np.complex128)
    got = _run_gh(3, 2, 1, [(0.9, 0.5)], s, T / n, 2, renorm=2, psi0=psi0)[0]
    ref = O.evolve(lat, Couplings(0.9, 0.5), s, T / n, 2, psi0=psi0)
    rel, mx = _rel(got, ref / np.linalg.norm(ref))
    assert rel <= 1e-10 and mx <= 1e-10, (rel, mx)


@gpu
def test_27_qubit_gauge_higgs_slice_matches_unitary_gauge_oracle():
    """3x3 torus, 27 qubits, complex128 double-float passes (plan 12 + 8 + 7, shared
    passes), 12 second-order steps: the tau = 0 slice times 2^{9/2} equals the 18-qubit
    unitary-gauge oracle run to 1e-10."""
    import torch
    from paper_2108_13410_gb300 import Simulator
    ug = OracleLattice(3, 3, True, "ug")
    s = O.schedule_linear(20.0, 1000)[:12]
    ref = O.evolve(ug, Couplings(0.6, 0.6), s, 0.02, 2)
    sim = Simulator(3, 3, form="gh", dtype="c128")
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, 0.02, 2)
    sl = sim.state[0, : 1 << 18].cpu().numpy() * 2 ** 4.5
    rel, mx = _rel(sl, ref)
    assert rel <= 1e-10 and mx <= 1e-10, (rel, mx)
    del sim
    torch.cuda.empty_cache()


@gpu
@pytest.mark.parametrize("lattice,form", [((2, 2), "gh"), ((3, 2), "ug"), ((4, 2), "ug")],
                         ids=["gh2x2open-21q", "ug3x2open-17q", "ug4x2open-22q"])
def test_open_lattices(lattice, form):
    """Open lattices with edge pass plans (12 + 8 + 1, 12 + 5, 12 + 8 + 2) in complex128
    double-float passes: oracle parity at 1e-10."""
    from paper_2108_13410_gb300 import Simulator
    Lx, Ly = lattice
    lat = OracleLattice(Lx, Ly, False, form)
    n_steps = 3
    T = 0.15 * n_steps
    s = O.schedule_linear(T, n_steps)
    ref = O.evolve(lat, Couplings(0.7, 0.4), s, T / n_steps, 2)
    sim = Simulator(Lx, Ly, form=form, dtype="c128", boundary="open")
    sim.init_plus()
    sim.evolve([(0.7, 0.4)], s, T / n_steps, 2)
    rel, mx = _rel(sim.download()[0].numpy(), ref)
    assert rel <= 1e-10 and mx <= 1e-10, (rel, mx)
