"""qs_dos against the oracle's density of states (Sec. V)."""
from math import comb

import numpy as np
import pytest

from oracle import OracleLattice, Couplings
from oracle import core as O

gpu = pytest.mark.gpu


@gpu
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-5)])
def test_dos_matches_oracle(dtype, tol):
    from paper_2108_13410_gb300 import Simulator
    lat = OracleLattice(3, 2, True, "gh")
    s = O.schedule_linear(3.0, 30)
    ref = O.dos(O.evolve(lat, Couplings(0.6, 0.2), s, 0.1, 2), lat)
    sim = Simulator(3, 2, form="gh", dtype=dtype)
    sim.init_plus()
    sim.evolve([(0.6, 0.2)], s, 0.1, 2)
    np.testing.assert_allclose(sim.dos()[0], ref, atol=tol)


@gpu
def test_dos_of_plus_state_at_32_qubits():
    from paper_2108_13410_gb300 import Simulator
    import torch
    sim = Simulator(4, 4, form="ug", dtype="c64")
    sim.init_plus()
    d = sim.dos()[0]
    np.testing.assert_allclose(d, [comb(32, k) / 2 ** 32 for k in range(33)], atol=1e-6)
    del sim
    torch.cuda.empty_cache()
