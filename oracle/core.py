"""Oracle for the Trotterised adiabatic evolution (test infrastructure only).

Composes the FP64 C primitives of qs_oracle.c one Pauli term at a time, in the
order the algorithm states:

* Hamiltonian.  Sec. II, Eq. (1) (gauge-Higgs form) and Eq. (4) (unitary-gauge
  form).  The adiabatic path interpolates H(s) = (1 - s) H0 + s H1 with H1 the
  model Hamiltonian and H0 = -sum of transverse fields, whose ground state |+>^n
  is the start of the path (Sec. III: the ground state is carried along a path
  in parameter space by many steps of equal duration).
    gauge-Higgs:     H0 = -sum_l sigma^x_l - sum_v tau^x_v
    unitary gauge:   H0 = -sum_l sigma^x_l - sum_v A^x_v   (the image of -sum tau^x
                     under Gauss's law Q_v = tau^x_v A^x_v = 1, Eq. (3))
* Groups.  All X-type terms (sigma^x, tau^x, A_v) commute with one another and all
  Z-type terms (B_p, tau^z sigma^z tau^z, sigma^z) commute with one another, so each
  group's exponential is an exact product of single-term factors (Eq. (8) and the
  remark after it).
* Trotter product.  Operators act right to left (end of Sec. III).  First order:
  U = exp(-i dt H_Z) exp(-i dt H_X) (X applied first).  Second order, Eq. (7):
  U = exp(-i dt/2 H_X) exp(-i dt H_Z) exp(-i dt/2 H_X); the paper's five-factor
  form reduces to this because the A_v half-factors commute with the sigma^x
  factors and the B_p half-factors commute with the sigma^z factor.
* Schedule.  Step k of N uses s_k = s(t_k) at the midpoint t_k = (k - 1/2) dt.

Nothing here fuses terms, caches phase tables or merges half-steps.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build
from .lattice import OracleLattice, mask_of

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        U = ctypes.c_uint64
        sig = {
            "or_init_plus": ([P, I], None),
            "or_apply_xrot": ([P, I, I, D], None),
            "or_apply_xstring": ([P, I, U, D], None),
            "or_apply_zphase": ([P, I, U, D], None),
            "or_axpy_xstring": ([P, P, I, U, D], None),
            "or_axpy_zstring": ([P, P, I, U, D], None),
            "or_inner": ([P, P, I, P, P], None),
            "or_expect_zstring": ([P, I, U], D),
            "or_expect_xstring": ([P, I, U], D),
            "or_xrot_tangent": ([P, P, I, P, I, I, D], None),
            "or_xstring_tangent": ([P, P, I, P, I, U, D], None),
            "or_zphase_tangent": ([P, P, I, P, I, U, D], None),
            "or_max_threads": ([], I),
            "or_set_threads": ([I], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---------------------------------------------------------------------------
# couplings and coefficients
# ---------------------------------------------------------------------------
class Couplings:
    """H1 couplings (J, h, g, lambda) of Eq. (1) / Eq. (4)."""

    def __init__(self, g: float, lam: float, J: float = 1.0, h: float = 1.0):
        self.J, self.h, self.g, self.lam = float(J), float(h), float(g), float(lam)

    def __repr__(self):
        return f"Couplings(J={self.J}, h={self.h}, g={self.g}, lam={self.lam})"


def coefficients(c: Couplings, s: float) -> dict:
    """Term coefficients of -H(s), H(s) = (1-s) H0 + s H1.

    x_sigma multiplies sigma^x_l, x_tau multiplies tau^x_v (gauge-Higgs) or A_v
    (unitary gauge), z_plaq multiplies B_p, z_second multiplies the bond
    tau^z sigma^z tau^z (gauge-Higgs) or sigma^z_l (unitary gauge).  H(s) is minus
    the sum of coefficient x term.
    """
    return dict(x_sigma=(1.0 - s) + s * c.g, x_tau=(1.0 - s) + s * c.J,
                z_plaq=s * c.h, z_second=s * c.lam)


def coefficient_derivatives(c: Couplings) -> dict:
    """d/ds of coefficients()."""
    return dict(x_sigma=c.g - 1.0, x_tau=c.J - 1.0, z_plaq=c.h, z_second=c.lam)


# ---------------------------------------------------------------------------
# states
# ---------------------------------------------------------------------------
def plus_state(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().or_init_plus(_p(psi), n)
    return psi


def _terms(lat: OracleLattice):
    """Ordered factor lists (kind, mask-or-qubit, coefficient key)."""
    xs = [("xrot", q, "x_sigma" if k == "s" else "x_tau") for q, k in lat.x_single()]
    xs += [("xstring", m, "x_tau") for m in lat.x_strings()]
    zs = [("zphase", m, "z_plaq") for m in lat.z_plaquettes()]
    zs += [("zphase", m, "z_second") for m in lat.z_second()]
    return xs, zs


def _apply(psi, n, kind, target, theta):
    L = lib()
    if kind == "xrot":
        L.or_apply_xrot(_p(psi), n, int(target), float(theta))
    elif kind == "xstring":
        L.or_apply_xstring(_p(psi), n, int(target), float(theta))
    else:
        L.or_apply_zphase(_p(psi), n, int(target), float(theta))


def apply_group(psi: np.ndarray, lat: OracleLattice, group: str, coef: dict, tau: float):
    """exp(-i tau H_group) as a product of single-term factors exp(i coef*tau*P)."""
    xs, zs = _terms(lat)
    for kind, target, key in (xs if group == "x" else zs):
        _apply(psi, lat.n_qubits, kind, target, coef[key] * tau)


def trotter_step(psi: np.ndarray, lat: OracleLattice, c: Couplings, s: float, dt: float,
                 order: int) -> None:
    """One Trotter step of H(s) over time dt, in place (Eq. (7))."""
    coef = coefficients(c, s)
    if order == 1:
        apply_group(psi, lat, "x", coef, dt)
        apply_group(psi, lat, "z", coef, dt)
    elif order == 2:
        apply_group(psi, lat, "x", coef, 0.5 * dt)
        apply_group(psi, lat, "z", coef, dt)
        apply_group(psi, lat, "x", coef, 0.5 * dt)
    else:
        raise ValueError("order must be 1 or 2")


def midpoints(T: float, n_steps: int) -> np.ndarray:
    dt = T / n_steps
    return (np.arange(1, n_steps + 1) - 0.5) * dt


def schedule_linear(T: float, n_steps: int) -> np.ndarray:
    """s_k = t_k / T at the step midpoints."""
    return midpoints(T, n_steps) / T


def schedule_fourier(T: float, n_steps: int, a) -> np.ndarray:
    """s(t) = t/T + sum_{m=1..M} a_m sin(m pi t / T) at the step midpoints."""
    t = midpoints(T, n_steps)
    s = t / T
    for m, am in enumerate(a, start=1):
        s = s + am * np.sin(m * math.pi * t / T)
    return s


def schedule_fourier_jacobian(T: float, n_steps: int, M: int) -> np.ndarray:
    """ds_k / da_m = sin(m pi t_k / T), shape (M, n_steps)."""
    t = midpoints(T, n_steps)
    return np.stack([np.sin(m * math.pi * t / T) for m in range(1, M + 1)])


def evolve(lat: OracleLattice, c: Couplings, s_list, dt: float, order: int,
           psi0: np.ndarray | None = None, callback=None) -> np.ndarray:
    psi = plus_state(lat.n_qubits) if psi0 is None else np.array(psi0, dtype=np.complex128)
    for k, s in enumerate(s_list):
        trotter_step(psi, lat, c, float(s), dt, order)
        if callback is not None:
            callback(k, psi)
    return psi


# ---------------------------------------------------------------------------
# observables (direct sums)
# ---------------------------------------------------------------------------
def norm2(psi):
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_inner(_p(psi), _p(psi), _nq(psi), ctypes.byref(re), ctypes.byref(im))
    return re.value


def _nq(psi):
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    return n


def inner(a, b):
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_inner(_p(a), _p(b), _nq(a), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def expect_z(psi, mask: int) -> float:
    return lib().or_expect_zstring(_p(psi), _nq(psi), int(mask))


def expect_x(psi, mask: int) -> float:
    return lib().or_expect_xstring(_p(psi), _nq(psi), int(mask))


def fidelity(phi, psi) -> float:
    return abs(inner(phi, psi)) ** 2


def energy(psi, lat: OracleLattice, c: Couplings, s: float = 1.0) -> float:
    """<psi|H(s)|psi> as the coefficient-weighted sum of single-term expectations."""
    coef = coefficients(c, s)
    e = 0.0
    for q, kind in lat.x_single():
        e -= coef["x_sigma" if kind == "s" else "x_tau"] * expect_x(psi, 1 << q)
    for m in lat.x_strings():
        e -= coef["x_tau"] * expect_x(psi, m)
    for m in lat.z_plaquettes():
        e -= coef["z_plaq"] * expect_z(psi, m)
    for m in lat.z_second():
        e -= coef["z_second"] * expect_z(psi, m)
    return e


def apply_hamiltonian(psi, lat: OracleLattice, c: Couplings, s: float = 1.0) -> np.ndarray:
    """H(s) psi built term by term."""
    coef = coefficients(c, s)
    out = np.zeros_like(psi)
    n = lat.n_qubits
    L = lib()
    for q, kind in lat.x_single():
        L.or_axpy_xstring(_p(out), _p(psi), n, 1 << q, -coef["x_sigma" if kind == "s" else "x_tau"])
    for m in lat.x_strings():
        L.or_axpy_xstring(_p(out), _p(psi), n, m, -coef["x_tau"])
    for m in lat.z_plaquettes():
        L.or_axpy_zstring(_p(out), _p(psi), n, m, -coef["z_plaq"])
    for m in lat.z_second():
        L.or_axpy_zstring(_p(out), _p(psi), n, m, -coef["z_second"])
    return out


def observables(psi, lat: OracleLattice, c: Couplings, s: float = 1.0) -> dict:
    return dict(
        norm=norm2(psi),
        energy=energy(psi, lat, c, s),
        plaquettes=[expect_z(psi, m) for m in lat.z_plaquettes()],
        wilson=[expect_z(psi, m) for m in lat.wilson()],
        x=[expect_x(psi, 1 << q) for q in range(lat.n_qubits)],
        gauss=[expect_x(psi, m) for m in lat.gauss()],
        thooft=[expect_x(psi, m) for m in lat.thooft()],
    )


# ---------------------------------------------------------------------------
# gradient by forward-mode tangents (a different algorithm from the adjoint)
# ---------------------------------------------------------------------------
def evolve_with_tangents(lat: OracleLattice, c: Couplings, s_list, dt: float, order: int,
                         ds_dp: np.ndarray, psi0: np.ndarray | None = None):
    """Evolve psi and d psi / d p for parameters p with ds_k/dp = ds_dp[p, k].

    Each factor exp(i theta P) with theta = coef(s_k) * tau gives
    d theta / d p = coef'(s_k) * tau * ds_dp[p, k].
    Returns (psi_N, dpsi_N) with dpsi of shape (P, 2^n)."""
    n = lat.n_qubits
    ds_dp = np.asarray(ds_dp, dtype=np.float64)
    P = ds_dp.shape[0]
    psi = plus_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    dpsi = np.zeros((P, 1 << n), dtype=np.complex128)
    dcoef = coefficient_derivatives(c)
    xs, zs = _terms(lat)
    L = lib()

    def group(terms, coef, tau, k):
        for kind, target, key in terms:
            theta = coef[key] * tau
            dth = np.ascontiguousarray(dcoef[key] * tau * ds_dp[:, k])
            fn = {"xrot": L.or_xrot_tangent, "xstring": L.or_xstring_tangent,
                  "zphase": L.or_zphase_tangent}[kind]
            fn(_p(psi), dpsi.ctypes.data, P, dth.ctypes.data, n, int(target), float(theta))

    for k, s in enumerate(s_list):
        coef = coefficients(c, float(s))
        if order == 1:
            group(xs, coef, dt, k)
            group(zs, coef, dt, k)
        else:
            group(xs, coef, 0.5 * dt, k)
            group(zs, coef, dt, k)
            group(xs, coef, 0.5 * dt, k)
    return psi, dpsi


def energy_gradient(lat, c, s_list, dt, order, ds_dp, psi0=None):
    """E = <psi_N|H1|psi_N> and dE/dp = 2 Re <dpsi_N|H1 psi_N>."""
    psi, dpsi = evolve_with_tangents(lat, c, s_list, dt, order, ds_dp, psi0)
    hpsi = apply_hamiltonian(psi, lat, c, 1.0)
    e = inner(psi, hpsi).real
    g = np.array([2.0 * inner(np.ascontiguousarray(d), hpsi).real for d in dpsi])
    return e, g


def fidelity_gradient(lat, c, s_list, dt, order, ds_dp, phi, psi0=None):
    """F = |<phi|psi_N>|^2 and dF/dp = 2 Re( conj(<phi|psi_N>) <phi|dpsi_N> )."""
    psi, dpsi = evolve_with_tangents(lat, c, s_list, dt, order, ds_dp, psi0)
    ov = inner(phi, psi)
    g = np.array([2.0 * (ov.conjugate() * inner(phi, np.ascontiguousarray(d))).real
                  for d in dpsi])
    return abs(ov) ** 2, g


def dos(psi, lat: OracleLattice) -> np.ndarray:
    """Density of states of Z~ = -sum_l sigma^z_l (Sec. V): weight of the eigenvalue
    Z~ = 2k - n_links, i.e. the sum of |psi_i|^2 over indices i with k link bits set."""
    links = lat.link_qubits
    out = np.zeros(len(links) + 1)
    p = np.abs(np.asarray(psi)) ** 2
    for i in range(p.size):
        k = sum((i >> q) & 1 for q in links)
        out[k] += p[i]
    return out


def evolve_path(lat: OracleLattice, path, dt: float, order: int, psi0: np.ndarray | None = None,
                callback=None) -> np.ndarray:
    """Parameter path (Sec. III): step k is a Trotter step of H1 with couplings path[k]
    (the Hamiltonian itself, s = 1)."""
    psi = plus_state(lat.n_qubits) if psi0 is None else np.array(psi0, dtype=np.complex128)
    for k, c in enumerate(path):
        trotter_step(psi, lat, c, 1.0, dt, order)
        if callback is not None:
            callback(k, psi)
    return psi


def toric_state(lat: OracleLattice, which: int) -> np.ndarray:
    """Toric-code ground states of Sec. IV, normalised.

    which = 0: psi_1 = prod_p (1 + B_p)/2 |+...+>   (Eq. (14): the plaquette projections)
    which = 1: psi_1' = prod_v (1 + A_v)/2 |0...0>  (Eq. (15): the star projections)
    Each projector (1 + P)/2 is applied term by term with the Pauli-string primitives."""
    n = lat.n_qubits
    L = lib()
    if which == 0:
        psi = plus_state(n)
        masks, axpy = lat.z_plaquettes(), L.or_axpy_zstring
    else:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
        masks, axpy = [mask_of(s) for s in lat.stars], L.or_axpy_xstring
    for m in masks:
        out = 0.5 * psi
        axpy(_p(out), _p(psi), n, int(m), 0.5)
        psi = out
    return psi / math.sqrt(norm2(psi))
