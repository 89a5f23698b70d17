"""Phase-diagram scan (qs_scan): every coupling point is an independent adiabatic
run; the observables per point match the oracle's run of that point.

Tolerances: observables of norm <= 1 within 1e-6 (complex128) and 3e-6 (complex64, about
3x the largest error measured on these cases, 1.0e-6); energies 1e-6 (complex128) and
1.2e-6 ||H|| (complex64, ||H|| <= the sum of |coefficients|; measured |dE| / ||H|| <= 3.5e-7,
the ratio of the parity tests).
"""
import numpy as np
import pytest

import synth
from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu


def _oracle_obs(lat, c, s, dt, order):
    psi = O.evolve(lat, c, s, dt, order)
    ob = O.observables(psi, lat, c, 1.0)
    links = lat.link_qubits
    sites = lat.site_qubits
    return np.array([ob["energy"], np.mean(ob["plaquettes"]),
                     ob["wilson"][0] if ob["wilson"] else 0.0, ob["wilson"][1] if ob["wilson"] else 0.0,
                     ob["norm"], np.mean([ob["x"][q] for q in links]),
                     np.mean([ob["x"][q] for q in sites]) if sites else 0.0, 0.0])


def _check(got, ref, dtype, hbound):
    obs_tol = 1e-6 if dtype == "c128" else 3e-6
    e_tol = 1e-6 if dtype == "c128" else 1.2e-6 * hbound
    assert abs(got[0] - ref[0]) <= e_tol, (got[0], ref[0])
    np.testing.assert_allclose(got[1:], ref[1:], atol=obs_tol)


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("order", [1, 2])
def test_scan_12_qubits_one_launch(dtype, order):
    from paper_2108_13410_gb300 import Simulator
    grid = synth.coupling_grid(4, 0.0, 1.5)           # 16 points on [0, 1.5]^2
    points = [tuple(p) for p in grid[::3]]             # 6 points
    T, n = 2.0, 20
    s = O.schedule_linear(T, n)
    sim = Simulator(2, 2, form="gh", dtype=dtype)
    out = sim.scan(points, s, T / n, order)
    lat = OracleLattice(2, 2, True, "gh")
    for k, (g, lam) in enumerate(points):
        c = Couplings(g, lam)
        ref = _oracle_obs(lat, c, s, T / n, order)
        _check(out[k], ref, dtype, 4 * 1.5 + 4 + 8 * 1.5 + 8 * 1.5)


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_scan_17_qubit_open_unitary_gauge_in_chunks(dtype):
    """3x2 plaquettes, open boundary, unitary gauge (17 link qubits); 6 points in
    chunks of 4 (the last chunk is padded)."""
    from paper_2108_13410_gb300 import Simulator
    points = [(0.1, 0.2), (0.5, 0.5), (1.0, 0.3), (0.3, 1.1), (1.4, 1.4), (0.0, 0.7)]
    T, n = 1.0, 8
    s = O.schedule_linear(T, n)
    sim = Simulator(3, 2, form="ug", dtype=dtype, boundary="open", batch=4)
    out = sim.scan(points, s, T / n, 2)
    lat = OracleLattice(3, 2, False, "ug")
    for k, (g, lam) in enumerate(points):
        ref = _oracle_obs(lat, Couplings(g, lam), s, T / n, 2)
        _check(out[k], ref, dtype, 17 * 1.5 + 12 + 6 + 17 * 1.5)


@gpu
def test_scan_point_equals_single_run():
    from paper_2108_13410_gb300 import Simulator, QS_PLAQUETTE
    T, n = 3.0, 30
    s = O.schedule_linear(T, n)
    sim = Simulator(2, 2, form="gh", dtype="c128")
    out = sim.scan([(0.6, 0.6), (0.2, 1.2)], s, T / n, 2)
    for k, cp in enumerate([(0.6, 0.6), (0.2, 1.2)]):
        sim.init_plus()
        sim.evolve([cp], s, T / n, 2)
        assert abs(sim.energy([cp])[0] - out[k, 0]) <= 1e-9
        assert abs(sim.expect(QS_PLAQUETTE, -1)[0] - out[k, 1]) <= 1e-9


@gpu
def test_scan_in_a_captured_graph_is_bit_identical():
    from paper_2108_13410_gb300 import Simulator, QS_OPT_GRAPH
    pts = [tuple(p) for p in synth.coupling_grid(4, 0.0, 1.5)]
    T, n = 2.0, 20
    s = O.schedule_linear(T, n)
    a = Simulator(2, 2, form="gh", dtype="c64")
    b = Simulator(2, 2, form="gh", dtype="c64")
    b.set_option(QS_OPT_GRAPH, 1)
    ra = a.scan(pts, s, T / n, 2)
    rb = b.scan(pts, s, T / n, 2)
    assert np.array_equal(ra, rb)
    # replay with other couplings and schedule values of the same shape
    pts2 = [(g + 0.05, l) for g, l in pts]
    s2 = O.schedule_linear(2 * T, n)
    assert np.array_equal(a.scan(pts2, s2, T / n, 2), b.scan(pts2, s2, T / n, 2))


# ---------------------------------------------------------------------------
# both lattices in one persistent launch (qs_scan_mixed)
# ---------------------------------------------------------------------------
MIX12 = [(0.2, 0.9), (0.6, 0.6), (1.3, 0.1)]
MIX17 = [(0.1, 0.2), (0.5, 0.5), (1.0, 0.3), (0.3, 1.1), (1.4, 1.4)]


def _mixed(order, slots=2, graph=False, n12=None, n17=None, T=1.0, n=8, buffers=0):
    from paper_2108_13410_gb300 import Simulator, QS_OPT_GRAPH
    from paper_2108_13410_gb300.qsim import qs_scan_mixed, QS_OPT_SCAN_BUFFERS
    p12 = MIX12 if n12 is None else MIX12[:n12]
    p17 = MIX17 if n17 is None else MIX17[:n17]
    s = O.schedule_linear(T, n)
    a = Simulator(2, 2, form="gh", dtype="c64")
    b = Simulator(3, 2, form="ug", dtype="c64", boundary="open", batch=slots)
    if graph:
        b.set_option(QS_OPT_GRAPH, 1)
    b.set_option(QS_OPT_SCAN_BUFFERS, buffers)
    return p12, p17, s, qs_scan_mixed(a.h, p12, b.h, p17, s, T / n, order)


@gpu
@pytest.mark.parametrize("order,buffers", [(1, 0), (2, 0), (2, 2), (2, 4), (2, 6)])
def test_mixed_scan_one_launch_matches_oracle(order, buffers):
    """Three 2x2 gauge-Higgs points and five 3x2-open unitary-gauge points (17 qubits) in
    one launch with two scratch slots, so CTAs take several points of both kinds from the
    queue and reuse their slot; every tile-buffer count of the 17-qubit passes."""
    p12, p17, s, (o12, o17) = _mixed(order, buffers=buffers)
    T, n = 1.0, 8
    lat12 = OracleLattice(2, 2, True, "gh")
    lat17 = OracleLattice(3, 2, False, "ug")
    for k, (g, lam) in enumerate(p12):
        _check(o12[k], _oracle_obs(lat12, Couplings(g, lam), s, T / n, order), "c64", 4 * 1.5 + 4 + 8 * 1.5 + 8 * 1.5)
    for k, (g, lam) in enumerate(p17):
        _check(o17[k], _oracle_obs(lat17, Couplings(g, lam), s, T / n, order), "c64", 17 * 1.5 + 12 + 6 + 17 * 1.5)


@gpu
def test_mixed_scan_single_lattice_and_graph_replay():
    """One lattice only (either), and a captured graph replays bit-identically."""
    _, p17, s, (o12, o17) = _mixed(2, n12=0)
    assert o12.shape == (0, 8) and o17.shape == (5, 8)
    _, _, _, (q12, q17) = _mixed(2)
    np.testing.assert_array_equal(o17, q17)            # results do not depend on the mix
    _, _, _, (r12, r17) = _mixed(2, n17=0)
    np.testing.assert_array_equal(r12, q12)
    _, _, _, (g12, g17) = _mixed(2, graph=True)
    np.testing.assert_array_equal(g12, q12)
    np.testing.assert_array_equal(g17, q17)


@gpu
def test_mixed_scan_rejects_wrong_lattices():
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300 import qsim as Q
    a = Simulator(2, 2, form="gh", dtype="c64")
    periodic = Simulator(3, 2, form="ug", dtype="c64", batch=1)          # 12 qubits: too small
    with pytest.raises(Q.QsError) as e:
        Q.qs_scan_mixed(a.h, MIX12, periodic.h, MIX17, [0.5], 0.1, 2)
    assert e.value.status == 1
    b = Simulator(3, 2, form="ug", dtype="c64", boundary="open", batch=1)
    c128 = Simulator(2, 2, form="gh", dtype="c128")
    with pytest.raises(Q.QsError) as e:
        Q.qs_scan_mixed(c128.h, MIX12, b.h, MIX17, [0.5], 0.1, 2)
    assert e.value.status == 1
