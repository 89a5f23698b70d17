"""Runtime features around the evolution: CUDA-graph replay, renormalisation,
checkpoint/resume and the device-side bounded wait (failure detection)."""
import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu


def _sim(*a, **k):
    from paper_2108_13410_gb300 import Simulator
    return Simulator(*a, **k)


@gpu
@pytest.mark.parametrize("form,L", [("gh", (3, 2)), ("ug", (2, 5))])
def test_graph_replay_is_bit_identical(form, L):
    from paper_2108_13410_gb300 import QS_OPT_GRAPH
    T, n = 2.0, 12
    s = O.schedule_linear(T, n)
    a = _sim(*L, form=form, dtype="c64")
    b = _sim(*L, form=form, dtype="c64")
    b.set_option(QS_OPT_GRAPH, 1)
    for sim in (a, b):
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, T / n, 2)
    assert np.array_equal(a.download().numpy(), b.download().numpy())
    # replay with a different schedule of the same length reuses the graph
    s2 = O.schedule_linear(2 * T, n)
    for sim in (a, b):
        sim.init_plus()
        sim.evolve([(0.3, 0.9)], s2, T / n, 2)
        sim.sync()
    assert np.array_equal(a.download().numpy(), b.download().numpy())


@gpu
def test_renormalisation_keeps_unit_norm_and_the_state():
    from paper_2108_13410_gb300 import QS_NORM
    lat = OracleLattice(3, 2, True, "gh")
    T, n = 4.0, 80
    s = O.schedule_linear(T, n)
    ref = O.evolve(lat, Couplings(0.6, 0.6), s, T / n, 2)
    sim = _sim(3, 2, form="gh", dtype="c64", renorm_every=10)
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, T / n, 2)
    assert abs(sim.expect(QS_NORM)[0] - 1.0) <= 1e-6
    got = sim.download()[0].numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 1e-5


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128", "c128-df"])
def test_checkpoint_resume_is_bit_identical(tmp_path, dtype):
    """Save after 9 of 20 first-order steps, load into a new simulator, finish: the
    state is bit-identical to the same two calls without the checkpoint.  Splitting
    the run into two calls is itself exact with separate FP64 passes (complex128 with
    QS_OPT_C128_DF 0); with shared passes (complex64, and complex128 in double-float
    passes, which also convert the layout at every call boundary) the first X factors
    of the second call meet their qubit groups in another order, which changes
    rounding only."""
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE, QS_OPT_C128_DF
    T, n = 2.0, 20
    s = O.schedule_linear(T, n)
    cpl = [(0.6, 0.6)]
    dt = "c64" if dtype == "c64" else "c128"

    def mk():
        sim = _sim(3, 2, form="gh", dtype=dt)
        if dtype == "c128":
            sim.set_option(QS_OPT_C128_DF, 0)
        return sim
    full = mk()
    full.init_plus()
    full.evolve(cpl, s, T / n, 1)
    two = mk()
    two.init_plus()
    two.evolve(cpl, s[:9], T / n, 1)
    two.evolve(cpl, s[9:], T / n, 1)
    part = mk()
    part.init_plus()
    part.evolve(cpl, s[:9], T / n, 1)
    path = str(tmp_path / "ckpt.qs")
    part.save(path)
    resumed = mk()
    resumed.load(path)
    resumed.evolve(cpl, s[9:], T / n, 1)
    assert np.array_equal(two.download().numpy(), resumed.download().numpy())
    a = full.download().numpy().astype(np.complex128)
    b = resumed.download().numpy().astype(np.complex128)
    if dtype == "c128":
        assert np.array_equal(a, b)
    elif dtype == "c128-df":
        assert np.linalg.norm(a - b) <= 1e-13
    else:
        assert np.linalg.norm(a - b) <= 1e-6
        # separate passes: the split is exact in complex64 too
        for sim in (full, part, resumed):
            sim.set_option(QS_OPT_XMERGE, 0)
        full.init_plus()
        full.evolve(cpl, s, T / n, 1)
        part.init_plus()
        part.evolve(cpl, s[:9], T / n, 1)
        path2 = str(tmp_path / "ckpt2.qs")
        part.save(path2)
        resumed.load(path2)
        resumed.evolve(cpl, s[9:], T / n, 1)
        assert np.array_equal(full.download().numpy(), resumed.download().numpy())
    other = _sim(2, 2, form="gh", dtype=dtype)
    from paper_2108_13410_gb300 import QsError
    with pytest.raises(QsError):
        other.load(path)


@gpu
def test_bounded_wait_times_out_and_the_context_survives():
    from paper_2108_13410_gb300 import QsError
    from paper_2108_13410_gb300.qsim import qs_selftest_wait
    sim = _sim(3, 2, form="gh", dtype="c64")
    with pytest.raises(QsError) as e:
        qs_selftest_wait(sim.h, 50.0)
    assert e.value.status == 5                     # QS_ERR_TIMEOUT
    # the context is still usable
    lat = OracleLattice(3, 2, True, "gh")
    s = O.schedule_linear(1.0, 5)
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, 0.2, 2)
    sim.sync()
    ref = O.evolve(lat, Couplings(0.6, 0.6), s, 0.2, 2)
    got = sim.download()[0].numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 1e-5


@gpu
def test_launch_count_is_reported():
    from paper_2108_13410_gb300.qsim import QS_OPT_XMERGE
    sim = _sim(3, 3, form="gh", dtype="c64")
    sim.init_plus()
    sim.launch_count()
    sim.evolve([(0.6, 0.6)], O.schedule_linear(1.0, 10), 0.1, 2)
    sim.sync()
    # device-built records (1) + 3 passes for the first factor group + 2 for each of
    # the other 10 (9 steps and the trailing X half): they share one pass each
    assert sim.launch_count() == 1 + 3 + 2 * 10
    sim.set_option(QS_OPT_XMERGE, 0)
    sim.evolve([(0.6, 0.6)], O.schedule_linear(1.0, 10), 0.1, 2)
    sim.sync()
    # separate passes: 3 x 10 steps + 3 trailing passes
    assert sim.launch_count() == 1 + 3 * 11


@gpu
def test_autotune_picks_a_valid_configuration(tmp_path, monkeypatch):
    monkeypatch.setenv("QSIM_CACHE", str(tmp_path / "tune.json"))
    sim = _sim(3, 3, form="gh", dtype="c64")
    e = sim.autotune(n_steps=4)
    assert e["xpass"] in (1, 2) and e["buffers"] in (2, 3) and e["store"] in (0, 1) and e["ms_per_step"] > 0
    assert e["shared_buffers"] in (0, 2, 3)          # 0: chosen by form
    again = sim.autotune(n_steps=4)           # from the cache
    keys = ("xpass", "buffers", "store", "shared_buffers")
    assert [again[k] for k in keys] == [e[k] for k in keys]
    # the chosen configuration still evolves correctly
    lat = OracleLattice(3, 3, True, "ug")
    s = O.schedule_linear(20.0, 1000)[:10]
    ref = O.evolve(lat, Couplings(0.6, 0.6), s, 0.02, 2)
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, 0.02, 2)
    sl = sim.state[0, : 1 << 18].cpu().numpy().astype(np.complex128) * 2 ** 4.5
    assert np.linalg.norm(sl - ref) <= 1e-5


@gpu
def test_energy_from_tiled_x_measurement_matches_oracle():
    """QS_ENERGY uses the read-only tiled X sweep for n >= 12; check it on 18 qubits against
    the oracle's term-by-term energy, and on 27 qubits against the 18-qubit unitary-gauge
    oracle (a gauge-invariant gauge-Higgs state has the energy of its unitary-gauge image)."""
    lat = OracleLattice(3, 2, True, "gh")
    s = O.schedule_linear(2.0, 20)
    ref = O.evolve(lat, Couplings(0.9, 0.4), s, 0.1, 2)
    # complex64: measured 3.0e-6 (s = 1) and 2.6e-6 (s = 0.3)
    for dtype, tol in (("c128", 1e-9), ("c64", 1e-5)):
        sim = _sim(3, 2, form="gh", dtype=dtype)
        sim.init_plus()
        sim.evolve([(0.9, 0.4)], s, 0.1, 2)
        assert abs(sim.energy([(0.9, 0.4)])[0] - O.energy(ref, lat, Couplings(0.9, 0.4))) <= tol
        assert abs(sim.energy([(0.9, 0.4)], s=0.3)[0] - O.energy(ref, lat, Couplings(0.9, 0.4), 0.3)) <= tol

    ug = OracleLattice(3, 3, True, "ug")
    s27 = O.schedule_linear(20.0, 1000)[:10]
    ref27 = O.evolve(ug, Couplings(0.6, 0.6), s27, 0.02, 2)
    sim = _sim(3, 3, form="gh", dtype="c64")
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s27, 0.02, 2)
    # complex64 after 10 steps: measured 7.0e-6
    assert abs(sim.energy([(0.6, 0.6)])[0] - O.energy(ref27, ug, Couplings(0.6, 0.6))) <= 3e-5


@gpu
@pytest.mark.parametrize("form,L", [("gh", (3, 3)), ("ug", (3, 3))])
def test_programmatic_dependent_launch_changes_nothing(form, L):
    """QS_OPT_PDL only lets an X pass be scheduled while the previous kernel drains (it
    waits for that kernel's writes before reading global memory): results with and without
    it are bit-identical, with renormalisation kernels in between."""
    from paper_2108_13410_gb300 import QS_OPT_RENORM_EVERY
    from paper_2108_13410_gb300.qsim import QS_OPT_PDL
    s = O.schedule_linear(2.0, 40)
    out = []
    for pdl in (1, 0):
        sim = _sim(*L, form=form, dtype="c64")
        sim.set_option(QS_OPT_PDL, pdl)
        sim.set_option(QS_OPT_RENORM_EVERY, 7)
        sim.init_plus()
        sim.evolve([(0.6, 0.6)], s, 0.05, 2)
        out.append(sim.download().numpy())
    assert np.array_equal(out[0], out[1])
