"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws random numbers and names workload sizes.  It holds none of
the method's arithmetic (no Hamiltonian, no Trotter factor, no schedule
evaluation): every quantity that the evolution computes is computed separately by
the CUDA path and by the oracle.

Workloads follow the five lattice set-ups studied for the Z2 gauge-Higgs model
(Sec. II, Sec. III): 2x2 and 3x3 periodic lattices in the gauge-Higgs form, a
3x2 open lattice and a 4x4 periodic lattice in the unitary-gauge form.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 2108


def rng(seed: int = DEFAULT_SEED) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_state(n_qubits: int, seed: int = DEFAULT_SEED, batch: int = 1) -> np.ndarray:
    """Complex Gaussian amplitudes, each batch row scaled to unit 2-norm (complex128)."""
    g = rng(seed)
    dim = 1 << n_qubits
    z = g.standard_normal((batch, dim)) + 1j * g.standard_normal((batch, dim))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return z if batch > 1 else z[0]


def random_angles(k: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Uniform angles in [-pi, pi]."""
    return rng(seed).uniform(-np.pi, np.pi, size=k)


def fourier_coeffs(m: int = 16, seed: int = DEFAULT_SEED, std: float = 0.01) -> np.ndarray:
    """Schedule perturbation amplitudes a_m ~ N(0, std^2), m = 1..M."""
    return rng(seed).normal(0.0, std, size=m)


def coupling_grid(points: int = 32, lo: float = 0.0, hi: float = 1.5) -> np.ndarray:
    """(g, lambda) pairs on a uniform points x points grid, endpoints included.

    Row-major: index = i * points + j holds (g_i, lambda_j)."""
    axis = np.linspace(lo, hi, points)
    g, lam = np.meshgrid(axis, axis, indexing="ij")
    return np.stack([g.ravel(), lam.ravel()], axis=1)


# Workload sizes (lattice, boundary, form, total time, steps, Trotter order).
WORKLOADS = {
    # 2x2 periodic gauge-Higgs: 8 link + 4 site qubits, first order, per-gate
    "gh2x2": dict(Lx=2, Ly=2, periodic=True, form="gh", T=10.0, steps=100, order=1,
                  couplings=[(0.2, 0.2), (0.6, 0.6), (1.2, 1.2)]),
    # 3x3 periodic gauge-Higgs: 18 link + 9 site = 27 qubits, second order
    "gh3x3": dict(Lx=3, Ly=3, periodic=True, form="gh", T=20.0, steps=1000, order=2,
                  couplings=[(0.2, 0.2), (0.6, 0.6), (1.2, 1.2)]),
    # batched scan: 2x2 gauge-Higgs (12 q) and 3x2 open unitary gauge (17 q)
    "scan": dict(points=32, lo=0.0, hi=1.5, T=10.0, steps=200, order=2),
    # adjoint gradient on 3x3 gauge-Higgs with a 16-term Fourier schedule
    "adjoint": dict(Lx=3, Ly=3, periodic=True, form="gh", T=20.0, steps=500, order=2,
                    M=16, couplings=[(0.6, 0.6)]),
    # 4x4 periodic unitary gauge: 32 link qubits
    "ug4x4": dict(Lx=4, Ly=4, periodic=True, form="ug", T=20.0, steps=1000, order=2,
                  couplings=[(0.5, 0.5)]),
}
