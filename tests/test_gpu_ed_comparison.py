"""Sec. VII: the Trotterised adiabatic evolution against exact diagonalisation on the
2x2 torus (unitary gauge, J = h = 1/2, the paper's parameters), along O(0,0) -> P(0.5, 0)
starting from the toric-code state psi_1.

The GPU energies along the path equal the oracle's (parity), and lie above the ED ground
energy of H1(g) at every checkpoint, within the adiabatic/Trotter excess (< 2e-2 here);
the curvature d^2E/dg^2 of the GPU curve follows the ED curve.
"""
import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O
from oracle import ed

gpu = pytest.mark.gpu


@gpu
def test_energy_along_o_to_p_matches_oracle_and_ed():
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.protocol import prepare, run_path
    lat = OracleLattice(2, 2, True, "ug")
    dg, dt = 1e-3, 0.05
    path = prepare(0.5, dg, "g")                         # 500 steps
    sim = Simulator(2, 2, form="ug", dtype="c128")
    sim.init_toric(0)
    got = run_path(sim, path, dt, 2, measure_every=25)
    checkpoints = {}

    def cb(k, psi):
        if (k + 1) % 25 == 0 or k + 1 == len(path):
            g, l, J, h = path[k]
            checkpoints[k] = O.energy(psi, lat, Couplings(g, l, J=J, h=h))

    O.evolve_path(lat, [Couplings(g, l, J=J, h=h) for g, l, J, h in path], dt, 2,
                  psi0=O.toric_state(lat, 0), callback=cb)
    ref = [checkpoints[k] for k in sorted(checkpoints)]
    e_gpu = np.array([e for _, e in got])
    np.testing.assert_allclose(e_gpu, ref, atol=1e-9)
    gs = np.array([c[0] for c, _ in got])
    e0 = np.array([ed.ground_energy(lat, Couplings(g, 0.0, J=0.5, h=0.5), 1.0)[0] for g in gs])
    assert np.all(e_gpu >= e0 - 1e-9)
    assert np.max(e_gpu - e0) < 2e-2
    # second derivative on the checkpoint grid (uniform spacing 25 * dg)
    h = gs[1] - gs[0]
    d2_gpu = np.diff(e_gpu, 2) / h ** 2
    d2_ed = np.diff(e0, 2) / h ** 2
    assert np.max(np.abs(d2_gpu - d2_ed)) < 0.5 * np.max(np.abs(d2_ed)) + 1.0
