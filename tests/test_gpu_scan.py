"""Phase-diagram scan (qs_scan): every coupling point is an independent adiabatic
run; the observables per point match the oracle's run of that point.

Tolerances as in the parity tests: observables of norm <= 1 within 1e-6 (complex128)
and 2e-5 (complex64); energies 1e-6 (complex128) and 2 ||H|| 1e-5 (complex64).
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
    obs_tol = 1e-6 if dtype == "c128" else 2e-5
    e_tol = 1e-6 if dtype == "c128" else 2 * hbound * 1e-5
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
