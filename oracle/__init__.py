"""FP64 CPU oracle for the Trotterised adiabatic evolution of the Z2 gauge-Higgs model.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  It shares no
code, tables or helpers with the CUDA path (paper_2108_13410_gb300); the only
code both sides use is the seeded input generator module `synth`.

Contents
  lattice.py   -- the oracle's own lattice numbering and Pauli term lists (Sec. II)
  qs_oracle.c  -- plain FP64 loops, one Pauli factor at a time (Eq. (7)-(8))
  core.py      -- Trotter steps, schedules, observables, forward-mode gradients
  ed.py        -- exact diagonalisation / exact propagators (Sec. VII, Appendix)
  bound.py     -- the Trotter error-bound arithmetic (Sec. VI, Appendix)

Parity pins: every function above is checked by tests/test_oracle_*.py against
dense Pauli matrices, exact diagonalisation, closed forms, invariants and the
numbers printed in Table I.  None is unpinned.
"""
from .lattice import OracleLattice, mask_of  # noqa: F401
from .core import (Couplings, coefficients, plus_state, trotter_step, evolve,  # noqa: F401
                   schedule_linear, schedule_fourier, schedule_fourier_jacobian,
                   energy, observables, expect_x, expect_z, norm2, inner, fidelity,
                   apply_hamiltonian, energy_gradient, fidelity_gradient,
                   evolve_with_tangents, set_threads, max_threads, dos,
                   evolve_path, toric_state)
