"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (the stated accuracy targets of the build):
  amplitudes: ||psi - psi_ref|| / ||psi_ref|| <= 1e-10 (complex128), 1e-5 (complex64),
              and max_i |psi_i - psi_ref_i| <= tol * max_i |psi_ref_i|;
  observables bounded by 1 (plaquettes, Wilson and 't Hooft loops, <X>, <Q_v>):
              1e-6 (complex128); 2e-6 (complex64: about 3x the largest error measured
              on these cases, 5.5e-7);
  energies:   1e-6 absolute (complex128); complex64 1.2e-6 ||H|| with ||H|| <= the sum
              of |coefficients| (the largest measured |dE| / ||H|| is 4e-7, on the
              24-qubit unitary-gauge torus; 1e-7 to 2e-7 on these cases).
  The complex64 bounds are set from measured errors so that a regression of a few
  times in accuracy fails; the rigorous bound |d<P>| <= 2 ||P|| ||d psi|| with
  ||d psi|| <= 1e-5 would hide a hundredfold one.
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


def _amp_tol(dtype):
    return 1e-10 if dtype == "c128" else 1e-5


def _assert_amplitudes(got, ref, dtype):
    got = np.asarray(got, dtype=np.complex128)
    tol = _amp_tol(dtype)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert rel <= tol and mx <= tol, (rel, mx, tol)


def _h_norm_bound(lat, c, s=1.0):
    coef = O.coefficients(c, s)
    nx = len(lat.link_qubits)
    return (nx * abs(coef["x_sigma"]) + (len(lat.site_qubits) + len(lat.x_strings())) * abs(coef["x_tau"])
            + len(lat.z_plaquettes()) * abs(coef["z_plaq"]) + len(lat.z_second()) * abs(coef["z_second"]))


C64_OBS_TOL = 2e-6
C64_ENERGY_PER_NORM = 1.2e-6
C64_NORM_TOL = 1e-6        # measured |<psi|psi> - 1| <= 2.3e-7


def _obs_tol(dtype):
    return 1e-6 if dtype == "c128" else C64_OBS_TOL


def _energy_tol(dtype, lat, c):
    return 1e-6 if dtype == "c128" else C64_ENERGY_PER_NORM * _h_norm_bound(lat, c)


def _run_oracle(lat, c, s, dt, order):
    return O.evolve(lat, c, s, dt, order)


CASES = [
    # (Lx, Ly, periodic, form, dtype, method, T, steps, order)
    (2, 2, True, "gh", "c128", "pergate", 10.0, 100, 1),   # the 12-qubit workload, per-gate
    (2, 2, True, "gh", "c128", "fused", 10.0, 100, 1),
    (2, 2, True, "gh", "c64", "fused", 10.0, 100, 1),
    (3, 2, True, "gh", "c128", "fused", 2.0, 20, 2),       # 18 qubits: 64 tiles, ragged 2nd pass
    (3, 2, True, "gh", "c64", "fused", 2.0, 20, 2),
    (3, 2, True, "gh", "c128", "pergate", 2.0, 10, 2),
    (3, 2, False, "ug", "c128", "fused", 2.0, 10, 2),      # 17-qubit open unitary gauge
    (3, 2, False, "ug", "c64", "fused", 2.0, 10, 2),
    (2, 2, True, "ug", "c128", "fused", 2.0, 20, 2),       # 8 qubits: smaller than one tile
]


@gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d%s-%s-%s-%s-o%d" % (
    c[0], c[1], "p" if c[2] else "o", c[3], c[4], c[5], c[8]))
def test_evolution_matches_oracle(case):
    Lx, Ly, periodic, form, dtype, method, T, n, order = case
    lat = OracleLattice(Lx, Ly, periodic, form)
    c = Couplings(0.6, 0.6)
    s = O.schedule_linear(T, n)
    ref = _run_oracle(lat, c, s, T / n, order)
    sim = _sim(Lx, Ly, form=form, dtype=dtype, boundary="periodic" if periodic else "open",
               method=method)
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, T / n, order)
    got = sim.download()[0].numpy()
    _assert_amplitudes(got, ref, dtype)
    # observables
    obs = O.observables(ref, lat, c, 1.0)
    e = sim.energy([(0.6, 0.6)])[0]
    assert abs(e - obs["energy"]) <= _energy_tol(dtype, lat, c)
    from paper_2108_13410_gb300 import QS_PLAQUETTE, QS_WILSON, QS_X, QS_GAUSS, QS_NORM
    tol = _obs_tol(dtype)
    for p, v in enumerate(obs["plaquettes"]):
        assert abs(sim.expect(QS_PLAQUETTE, p)[0] - v) <= tol
    for w, v in enumerate(obs["wilson"]):
        assert abs(sim.expect(QS_WILSON, w)[0] - v) <= tol
    for q in (0, lat.n_qubits - 1):
        assert abs(sim.expect(QS_X, q)[0] - obs["x"][q]) <= tol
    for v_, val in enumerate(obs["gauss"]):
        assert abs(sim.expect(QS_GAUSS, v_)[0] - val) <= tol
    assert abs(sim.expect(QS_NORM)[0] - 1.0) <= (1e-12 if dtype == "c128" else C64_NORM_TOL)


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_elements_are_independent_runs(dtype):
    couplings = [(0.2, 0.2), (0.6, 0.6), (1.2, 1.2)]
    T, n = 2.0, 10
    s = O.schedule_linear(T, n)
    simb = _sim(3, 2, form="gh", dtype=dtype, batch=3)
    simb.init_plus()
    simb.evolve(couplings, s, T / n, 2)
    got = simb.download().numpy()
    lat = OracleLattice(3, 2, True, "gh")
    for b, (g, lam) in enumerate(couplings):
        ref = _run_oracle(lat, Couplings(g, lam), s, T / n, 2)
        _assert_amplitudes(got[b], ref, dtype)
    es = simb.energy(couplings)
    for b, (g, lam) in enumerate(couplings):
        c = Couplings(g, lam)
        ref = _run_oracle(lat, c, s, T / n, 2)
        assert abs(es[b] - O.energy(ref, lat, c)) <= _energy_tol(dtype, lat, c)


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_trotter_step_equals_evolve_of_one_step(dtype):
    lat = OracleLattice(3, 2, True, "gh")
    c = Couplings(0.6, 0.6)
    sim = _sim(3, 2, form="gh", dtype=dtype)
    for order in (1, 2):
        sim.init_plus()
        sim.trotter_step([(0.6, 0.6)], 0.37, 0.11, order)
        ref = O.plus_state(lat.n_qubits)
        O.trotter_step(ref, lat, c, 0.37, 0.11, order)
        _assert_amplitudes(sim.download()[0].numpy(), ref, dtype)


@gpu
def test_fidelity_and_random_state_upload():
    import torch
    lat = OracleLattice(3, 2, True, "gh")
    psi0 = synth.random_state(lat.n_qubits, seed=21)
    phi = synth.random_state(lat.n_qubits, seed=22)
    sim = _sim(3, 2, form="gh", dtype="c128")
    sim.upload(torch.from_numpy(psi0.reshape(1, -1)).pin_memory())
    c = Couplings(0.9, 0.3)
    s = O.schedule_linear(1.0, 5)
    sim.evolve([(0.9, 0.3)], s, 0.2, 2)
    ref = O.evolve(lat, c, s, 0.2, 2, psi0=psi0)
    _assert_amplitudes(sim.download()[0].numpy(), ref, "c128")
    phi_dev = torch.from_numpy(phi.reshape(1, -1)).cuda()
    f = sim.fidelity(phi_dev)[0]
    assert abs(f - O.fidelity(phi, ref)) <= 1e-12


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_x_layer_closed_form_at_27_qubits(dtype):
    """h = lambda = 0: one first-order step is prod_q exp(i theta_q X_q) applied to
    |0...0>, whose amplitudes are prod_q (bit_q(i) ? i sin theta_q : cos theta_q)."""
    import torch
    sim = _sim(3, 3, form="gh", dtype=dtype)
    n = sim.n
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    zero = torch.zeros((1, 1 << n), dtype=tdt, pin_memory=True)
    zero[0, 0] = 1.0
    sim.upload(zero)
    s, dt, g, J = 0.4, 0.23, 0.7, 1.9
    sim.trotter_step([(g, 0.0, J, 0.0)], s, dt, 1)
    th_link = ((1 - s) + s * g) * dt
    th_site = ((1 - s) + s * J) * dt
    got = sim.download()[0].numpy()
    amax = np.cos(th_link) ** 18 * np.cos(th_site) ** 9      # the largest amplitude, at i = 0
    rng = np.random.default_rng(5)
    idx = np.concatenate([np.arange(64), rng.integers(0, 1 << n, 4000), [(1 << n) - 1]])
    for i in idx:
        i = int(i)
        nl = bin(i & ((1 << 18) - 1)).count("1")
        ns = bin(i >> 18).count("1")
        want = (np.cos(th_link) ** (18 - nl) * (1j * np.sin(th_link)) ** nl
                * np.cos(th_site) ** (9 - ns) * (1j * np.sin(th_site)) ** ns)
        assert abs(got[i] - want) <= _amp_tol(dtype) * amax
    norm = sim.expect(0)[0]
    assert abs(norm - 1.0) <= (1e-12 if dtype == "c128" else 2e-6)


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_z_layer_closed_form_at_27_qubits(dtype):
    """g = J = 0 at s = 1: the X angles vanish and one first-order step multiplies
    amplitude i by exp(i dt [h sum_p (-1)^{pi_p(i)} + lambda sum_b (-1)^{pi_b(i)}])."""
    import torch
    lat = OracleLattice(3, 3, True, "gh")
    n = lat.n_qubits
    sim = _sim(3, 3, form="gh", dtype=dtype)
    sim.init_plus()
    h, lam, dt = 0.8, 1.3, 0.07
    sim.trotter_step([(0.0, lam, 0.0, h)], 1.0, dt, 1)
    got = sim.download()[0].numpy()
    rng = np.random.default_rng(6)
    idx = np.concatenate([np.arange(32), rng.integers(0, 1 << n, 4000)])
    a = 2 ** (-n / 2)
    for i in idx:
        i = int(i)
        ph = h * sum(1 - 2 * (bin(i & m).count("1") & 1) for m in lat.z_plaquettes())
        ph += lam * sum(1 - 2 * (bin(i & m).count("1") & 1) for m in lat.z_second())
        want = a * np.exp(1j * dt * ph)
        assert abs(got[i] - want) <= _amp_tol(dtype) * a * 4


@gpu
def test_gauge_higgs_27_qubits_matches_unitary_gauge_oracle():
    """The tau = 0 slice of the 27-qubit gauge-Higgs run equals the 18-qubit
    unitary-gauge oracle run, psi_UG = 2^{9/2} psi_GH(sigma, tau = 0)."""
    ug = OracleLattice(3, 3, True, "ug")
    c = Couplings(0.6, 0.6)
    T, n = 20.0, 1000
    steps = 40
    s = O.schedule_linear(T, n)[:steps]
    ref = O.evolve(ug, c, s, T / n, 2)
    for dtype in ("c128", "c64"):
        sim = _sim(3, 3, form="gh", dtype=dtype)
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, T / n, 2)
        sl = sim.state[0, : 1 << 18].cpu().numpy().astype(np.complex128) * 2 ** 4.5
        _assert_amplitudes(sl, ref, dtype)
        del sim


@gpu
def test_errors_are_reported():
    from paper_2108_13410_gb300 import qsim as Q
    h = Q.qs_create(2, 2)
    with pytest.raises(Q.QsError) as e:
        Q.qs_init_plus(h)
    assert e.value.status == 6      # QS_ERR_STATE: nothing bound
    Q.qs_destroy(h)
    with pytest.raises(Q.QsError):
        Q.qs_create(1, 1)           # periodic lattice needs L >= 2
    sim = _sim(2, 2, form="gh", dtype="c64")
    sim.init_plus()
    with pytest.raises(Q.QsError):
        sim.trotter_step([(0.6, 0.6)], 0.5, 0.1, 3)   # order 3
    sim.state[0, 5] = float("nan")
    with pytest.raises(Q.QsError) as e:
        sim.expect(0)
    assert e.value.status == 4      # QS_ERR_NONFINITE


@gpu
@pytest.mark.parametrize("impl,nbuf,store", [(1, 2, 0), (2, 2, 0), (2, 3, 0), (2, 2, 1), (2, 3, 1)])
@pytest.mark.parametrize("form", ["ug", "gh"])
def test_complex64_xpass_kernels_agree(impl, nbuf, store, form):
    """The register-staged and the persistent TMA X-pass kernels (2 or 3 tile
    buffers, per-thread or bulk tensor stores) give the oracle's amplitudes on a
    20-qubit unitary-gauge and an 18-qubit gauge-Higgs lattice with batch 2."""
    from paper_2108_13410_gb300 import QS_OPT_XPASS, QS_OPT_TMA_BUFFERS
    from paper_2108_13410_gb300.qsim import QS_OPT_TMA_STORE
    if form == "gh":
        lat = OracleLattice(3, 2, True, "gh")
        couplings = [(0.6, 0.6), (1.1, 0.3)]
        s = O.schedule_linear(2.0, 12)
        sim = _sim(3, 2, form="gh", dtype="c64", batch=2)
        sim.set_option(QS_OPT_XPASS, impl)
        sim.set_option(QS_OPT_TMA_BUFFERS, nbuf)
        sim.set_option(QS_OPT_TMA_STORE, store)
        sim.init_plus()
        sim.evolve(couplings, s, 2.0 / 12, 2)
        sim.sync()
        got = sim.download().numpy()
        for b, (g, lam) in enumerate(couplings):
            _assert_amplitudes(got[b], O.evolve(lat, Couplings(g, lam), s, 2.0 / 12, 2), "c64")
        return
    lat = OracleLattice(2, 5, True, "ug")          # 20 link qubits, 256 tiles per state
    couplings = [(0.6, 0.6), (1.1, 0.3)]
    T, n = 2.0, 12
    s = O.schedule_linear(T, n)
    sim = _sim(2, 5, form="ug", dtype="c64", batch=2)
    sim.set_option(QS_OPT_XPASS, impl)
    sim.set_option(QS_OPT_TMA_BUFFERS, nbuf)
    sim.set_option(QS_OPT_TMA_STORE, store)
    sim.init_plus()
    sim.evolve(couplings, s, T / n, 2)
    sim.sync()
    got = sim.download().numpy()
    for b, (g, lam) in enumerate(couplings):
        ref = O.evolve(lat, Couplings(g, lam), s, T / n, 2)
        _assert_amplitudes(got[b], ref, "c64")


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_unitary_gauge_4x4_32_qubits(dtype):
    """4x4 torus in the unitary gauge: 32 link qubits (32 GB complex64, 64 GB complex128).
    One first-order step from |+>: |+> is an eigenstate of every X-type term (sigma^x
    and A_v, eigenvalue +1), so the X layer is the global phase exp(i(th_s N_l + th_t N_v))
    and amplitude i ends as 2^{-n/2} exp(i(th_s N_l + th_t N_v)) exp(i phi_Z(i)).
    Then further second-order steps keep the norm, lattice symmetry and, at lambda = 0,
    the 't Hooft loops."""
    from paper_2108_13410_gb300 import QS_NORM, QS_PLAQUETTE, QS_THOOFT, QS_X
    import torch
    lat = OracleLattice(4, 4, True, "ug")
    n = lat.n_qubits
    g, lam, s, dt = 0.5, 0.0, 0.7, 0.05
    sim = _sim(4, 4, form="ug", dtype=dtype)
    sim.init_plus()
    sim.trotter_step([(g, lam)], s, dt, 1)
    coef = O.coefficients(Couplings(g, lam), s)
    glob = coef["x_sigma"] * dt * 32 + coef["x_tau"] * dt * 16
    rng = np.random.default_rng(9)
    idx = rng.integers(0, 1 << n, 512)
    amp = sim.state[0, torch.from_numpy(idx).to(sim.state.device)].cpu().numpy()
    a = 2 ** (-n / 2)
    for i, got in zip(idx, amp):
        i = int(i)
        ph = coef["z_plaq"] * sum(1 - 2 * (bin(i & m).count("1") & 1) for m in lat.z_plaquettes())
        ph += coef["z_second"] * sum(1 - 2 * (bin(i & m).count("1") & 1) for m in lat.z_second())
        want = a * np.exp(1j * (glob + dt * ph))
        assert abs(got - want) <= _amp_tol(dtype) * a * 4
    sim.evolve([(g, lam)], [0.2, 0.4, 0.6], 0.1, 2)
    assert abs(sim.expect(QS_NORM)[0] - 1.0) <= (1e-10 if dtype == "c128" else 1e-5)
    pl = [sim.expect(QS_PLAQUETTE, p)[0] for p in (0, 5, 15)]
    assert max(pl) - min(pl) <= _obs_tol(dtype)
    xs = [sim.expect(QS_X, q)[0] for q in (0, 17, 31)]
    assert max(xs) - min(xs) <= _obs_tol(dtype)
    for k in (0, 1):
        assert abs(sim.expect(QS_THOOFT, k)[0] - 1.0) <= _obs_tol(dtype)
    del sim
    torch.cuda.empty_cache()
