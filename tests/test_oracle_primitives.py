"""Pins of the oracle's FP64 primitives against dense Pauli matrices.

The dense operators are built here from 2x2 Pauli matrices with numpy.kron and
exponentiated with scipy.linalg.expm, an algorithm independent of the
cos/sin closed form the oracle uses (exp(i theta P) = cos theta + i sin theta P).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import core

I2 = np.eye(2)
X2 = np.array([[0, 1], [1, 0]], dtype=complex)
Z2 = np.array([[1, 0], [0, -1]], dtype=complex)
N = 5


def pauli(n, mask, P):
    """kron over qubits n-1 .. 0 (qubit q <-> bit q of the amplitude index)."""
    out = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        out = np.kron(out, P if (mask >> q) & 1 else I2)
    return out


def state(seed):
    return np.ascontiguousarray(synth.random_state(N, seed=seed))


@pytest.mark.parametrize("q", range(N))
def test_xrot_matches_dense(q):
    psi = state(q)
    theta = 0.37 + 0.1 * q
    ref = sla.expm(1j * theta * pauli(N, 1 << q, X2)) @ psi
    core.lib().or_apply_xrot(psi.ctypes.data, N, q, theta)
    np.testing.assert_allclose(psi, ref, atol=1e-13)


@pytest.mark.parametrize("mask", [0b00011, 0b10110, 0b11111, 0b01000])
def test_xstring_matches_dense(mask):
    psi = state(mask)
    theta = -1.1
    ref = sla.expm(1j * theta * pauli(N, mask, X2)) @ psi
    core.lib().or_apply_xstring(psi.ctypes.data, N, mask, theta)
    np.testing.assert_allclose(psi, ref, atol=1e-13)


@pytest.mark.parametrize("mask", [0b00001, 0b01011, 0b11111, 0b10100])
def test_zphase_matches_dense(mask):
    psi = state(100 + mask)
    theta = 0.83
    ref = sla.expm(1j * theta * pauli(N, mask, Z2)) @ psi
    core.lib().or_apply_zphase(psi.ctypes.data, N, mask, theta)
    np.testing.assert_allclose(psi, ref, atol=1e-13)


def test_axpy_and_expectations_match_dense():
    psi = state(7)
    mx, mz = 0b10101, 0b01110
    PX, PZ = pauli(N, mx, X2), pauli(N, mz, Z2)
    out = np.zeros_like(psi)
    core.lib().or_axpy_xstring(out.ctypes.data, psi.ctypes.data, N, mx, 0.5)
    core.lib().or_axpy_zstring(out.ctypes.data, psi.ctypes.data, N, mz, -2.0)
    np.testing.assert_allclose(out, 0.5 * PX @ psi - 2.0 * PZ @ psi, atol=1e-13)
    assert core.expect_x(psi, mx) == pytest.approx(np.vdot(psi, PX @ psi).real, abs=1e-13)
    assert core.expect_z(psi, mz) == pytest.approx(np.vdot(psi, PZ @ psi).real, abs=1e-13)
    phi = state(8)
    assert core.inner(phi, psi) == pytest.approx(np.vdot(phi, psi), abs=1e-13)
    assert core.norm2(psi) == pytest.approx(1.0, abs=1e-13)


def test_plus_state():
    psi = core.plus_state(N)
    np.testing.assert_allclose(psi, np.full(1 << N, 2 ** (-N / 2)), atol=1e-15)


@pytest.mark.parametrize("kind", ["xrot", "xstring", "zphase"])
def test_tangent_primitives(kind):
    """d/da [exp(i theta(a) P) psi(a)] = exp(i theta P) psi' + theta' i P exp(i theta P) psi,
    checked with dense matrices for two tangents at once."""
    psi = state(11)
    d = np.ascontiguousarray(np.stack([state(12), state(13)]))
    theta = 0.71
    dth = np.array([0.3, -1.7])
    target = {"xrot": 1 << 2, "xstring": 0b11010, "zphase": 0b00111}[kind]
    P = pauli(N, target, Z2 if kind == "zphase" else X2)
    U = sla.expm(1j * theta * P)
    new_psi = U @ psi
    ref_d = [U @ d[k] + dth[k] * 1j * (P @ new_psi) for k in range(2)]
    L = core.lib()
    fn = {"xrot": L.or_xrot_tangent, "xstring": L.or_xstring_tangent,
          "zphase": L.or_zphase_tangent}[kind]
    tgt = 2 if kind == "xrot" else target
    fn(psi.ctypes.data, d.ctypes.data, 2, dth.ctypes.data, N, tgt, theta)
    np.testing.assert_allclose(psi, new_psi, atol=1e-13)
    np.testing.assert_allclose(d[0], ref_d[0], atol=1e-12)
    np.testing.assert_allclose(d[1], ref_d[1], atol=1e-12)
