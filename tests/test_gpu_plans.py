"""Pass plans of the tiled X layer (QS_OPT_PLAN, qs_plan, qs_autotune_plan).

A plan fixes how many new qubits each HBM pass after the first fuses (the first pass
always takes qubits 0..11); a pass fusing k new qubits keeps a contiguous chunk of
12 - k low qubits.  Every plan applies the same product of commuting X factors
(Eq. (8)), so the results agree with the oracle whatever the plan, up to rounding.
"""
import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu

T_P, N_P = 2.0, 8


@pytest.fixture(scope="module")
def oracle_3x4_ug():
    lat = OracleLattice(3, 4, True, "ug")
    s = O.schedule_linear(T_P, N_P)
    return lat, s, O.evolve(lat, Couplings(0.5, 0.5), s, T_P / N_P, 2)


def _rel(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref), np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@gpu
@pytest.mark.parametrize("plan", [[12, 4, 8], [12, 6, 6], [12, 8, 4], [12, 7, 5]])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_every_plan_matches_the_oracle_on_24_qubits(oracle_3x4_ug, plan, dtype):
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_PLAN, plan_code
    lat, s, ref = oracle_3x4_ug
    sim = Simulator(3, 4, form="ug", dtype=dtype)
    sim.set_option(QS_OPT_PLAN, plan_code(plan))
    assert sim.plan() == plan
    sim.init_plus()
    sim.evolve([(0.5, 0.5)], s, T_P / N_P, 2)
    rel, mx = _rel(sim.download()[0].numpy(), ref)
    tol = 1e-10 if dtype == "c128" else 1e-5
    assert rel <= tol and mx <= tol, (rel, mx)


@gpu
@pytest.mark.parametrize("plan", [[12, 8, 7], [12, 7, 8]])
def test_both_27_qubit_plans_match_the_unitary_gauge_oracle(plan):
    """The tau = 0 slice of the 27-qubit gauge-Higgs run equals the 18-qubit unitary-gauge
    oracle run (psi_UG = 2^{9/2} psi_GH(sigma, tau = 0)) with either plan, shared passes on."""
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import QS_OPT_PLAN, plan_code
    ug = OracleLattice(3, 3, True, "ug")
    s = O.schedule_linear(20.0, 1000)[:12]
    ref = O.evolve(ug, Couplings(0.6, 0.6), s, 0.02, 2)
    sim = Simulator(3, 3, form="gh", dtype="c64")
    sim.set_option(QS_OPT_PLAN, plan_code(plan))
    assert sim.plan() == plan
    sim.init_plus()
    sim.evolve([(0.6, 0.6)], s, 0.02, 2)
    sl = sim.state[0, : 1 << 18].cpu().numpy().astype(np.complex128) * 2 ** 4.5
    rel, mx = _rel(sl, ref)
    assert rel <= 1e-5 and mx <= 1e-5, (rel, mx)


@gpu
def test_plan_autotuner_picks_a_valid_plan(oracle_3x4_ug):
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.qsim import qs_autotune_plan
    lat, s, ref = oracle_3x4_ug
    sim = Simulator(3, 4, form="ug", dtype="c64")
    plan, ms = qs_autotune_plan(sim.h, 4)
    assert plan[0] == 12 and sum(plan) == 24 and len(plan) == 3 and all(4 <= k <= 8 for k in plan[1:])
    assert ms > 0.0 and sim.plan() == plan
    sim.init_plus()
    sim.evolve([(0.5, 0.5)], s, T_P / N_P, 2)
    rel, mx = _rel(sim.download()[0].numpy(), ref)
    assert rel <= 1e-5 and mx <= 1e-5


@gpu
def test_bad_plans_are_rejected():
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300 import qsim as Q
    sim = Simulator(3, 4, form="ug", dtype="c64")
    for bad in ([12, 8, 5], [12, 9, 3], [12, 12]):
        with pytest.raises(Q.QsError) as e:
            sim.set_option(Q.QS_OPT_PLAN, Q.plan_code(bad))
        assert e.value.status == 1
    assert sim.plan() == [12, 8, 4]                 # unchanged: the default plan
    small = Simulator(2, 2, form="gh", dtype="c64")  # 12 qubits: one tile, no plan
    with pytest.raises(Q.QsError):
        small.set_option(Q.QS_OPT_PLAN, Q.plan_code([12, 4]))
    assert small.plan() == [12]
