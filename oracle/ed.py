"""Exact diagonalisation and exact propagators (test infrastructure only).

Sec. VII compares the Trotterised simulation with exact diagonalisation on a
2x2 torus.  Here the same comparison is done on matrices assembled from the
oracle's own term lists:

* X string on mask m: the permutation |i> -> |i xor m>.
* Z string on mask m: diag((-1)^{popcount(i & m)}).

Used for: ground energies (variational bound of the adiabatic result), exact
piecewise-constant propagators prod_k exp(-i H(s_k) dt) (Trotter-order slopes),
dense group Hamiltonians and nested commutators (the second-order error bound of
the Appendix, taken from Childs et al.).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .core import Couplings, coefficients
from .lattice import OracleLattice


def _popcount_parity(idx: np.ndarray, mask: int) -> np.ndarray:
    x = idx & mask
    p = np.zeros_like(x)
    while True:
        nz = x != 0
        if not nz.any():
            break
        p ^= (x & 1)
        x >>= 1
    return p


def xstring_matrix(n: int, mask: int) -> sp.csr_matrix:
    dim = 1 << n
    idx = np.arange(dim, dtype=np.int64)
    return sp.csr_matrix((np.ones(dim), (idx ^ mask, idx)), shape=(dim, dim))


def zstring_diag(n: int, mask: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    return 1.0 - 2.0 * _popcount_parity(idx, mask)


def group_hamiltonians(lat: OracleLattice, c: Couplings, s: float):
    """(H_X, H_Z) sparse, with H(s) = H_X + H_Z."""
    n = lat.n_qubits
    dim = 1 << n
    coef = coefficients(c, s)
    hx = sp.csr_matrix((dim, dim))
    for q, kind in lat.x_single():
        hx = hx - coef["x_sigma" if kind == "s" else "x_tau"] * xstring_matrix(n, 1 << q)
    for m in lat.x_strings():
        hx = hx - coef["x_tau"] * xstring_matrix(n, m)
    dz = np.zeros(dim)
    for m in lat.z_plaquettes():
        dz -= coef["z_plaq"] * zstring_diag(n, m)
    for m in lat.z_second():
        dz -= coef["z_second"] * zstring_diag(n, m)
    return hx.tocsr(), sp.diags(dz).tocsr()


def hamiltonian(lat: OracleLattice, c: Couplings, s: float = 1.0) -> sp.csr_matrix:
    hx, hz = group_hamiltonians(lat, c, s)
    return (hx + hz).tocsr()


def gauss_sum(lat: OracleLattice) -> sp.csr_matrix:
    n = lat.n_qubits
    dim = 1 << n
    acc = sp.csr_matrix((dim, dim))
    for m in lat.gauss():
        acc = acc + xstring_matrix(n, m)
    return acc.tocsr()


def ground_energy(lat: OracleLattice, c: Couplings, s: float = 1.0, gauge_sector: bool = True,
                  k: int = 1) -> np.ndarray:
    """Lowest eigenvalues of H(s).  For the gauge-Higgs form with gauge_sector=True the
    spectrum is restricted to Q_v = +1 for every v (Gauss's law, Eq. (3)) by the exact
    shift H - mu * sum_v Q_v (the Q_v commute with H and with one another)."""
    H = hamiltonian(lat, c, s)
    shift = 0.0
    if gauge_sector and lat.form == "gh":
        mu = 10.0 * (lat.n_qubits + 4)
        H = H - mu * gauss_sum(lat)
        shift = mu * len(lat.gauss())
    dim = H.shape[0]
    if dim <= 4096:
        w = np.linalg.eigvalsh(H.toarray())[:k]
    else:
        w = np.sort(spla.eigsh(H, k=k, which="SA", tol=1e-12, maxiter=100000)[0])
    return w + shift


def exact_piecewise(lat: OracleLattice, c: Couplings, s_list, dt: float,
                    psi0: np.ndarray) -> np.ndarray:
    """prod_k exp(-i H(s_k) dt) psi0: the evolution that the Trotter product approximates."""
    psi = np.array(psi0, dtype=np.complex128)
    for s in s_list:
        H = hamiltonian(lat, c, float(s))
        psi = spla.expm_multiply(-1j * dt * H, psi)
    return psi


def dense(m) -> np.ndarray:
    return m.toarray() if sp.issparse(m) else np.asarray(m)


def spectral_norm(a: np.ndarray) -> float:
    return float(np.linalg.norm(a, 2))


def second_order_step_error(lat: OracleLattice, c: Couplings, s: float, dt: float,
                            s2: np.ndarray | None = None):
    """(||S_2(dt) - exp(-i H dt)||, Childs et al. bound) for the two-group split with the
    X group outermost: S_2 = e^{-i H_X dt/2} e^{-i H_Z dt} e^{-i H_X dt/2}.
    s2 may be supplied (e.g. assembled column by column from a step routine); by
    default it is built from dense exponentials of the group Hamiltonians.

    Bound (Appendix, Gamma = 2 groups, H_1 = H_X, H_2 = H_Z):
        dt^3/12 ||[H_2, [H_2, H_1]]|| + dt^3/24 ||[H_1, [H_1, H_2]]||."""
    hx, hz = group_hamiltonians(lat, c, s)
    A, B = dense(hx), dense(hz)
    if s2 is None:
        ux = sla.expm(-0.5j * dt * A)
        uz = sla.expm(-1j * dt * B)
        s2 = ux @ uz @ ux
    ex = sla.expm(-1j * dt * (A + B))
    err = spectral_norm(s2 - ex)

    def comm(x, y):
        return x @ y - y @ x

    bound = dt ** 3 / 12.0 * spectral_norm(comm(B, comm(B, A))) \
        + dt ** 3 / 24.0 * spectral_norm(comm(A, comm(A, B)))
    return err, bound
