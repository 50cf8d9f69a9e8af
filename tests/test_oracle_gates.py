"""Pins of the oracle's gate matrices against scipy's matrix exponential and
textbook identities (not the oracle's own formulas)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import gates as g

PAULI_TEXTBOOK = {
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


@pytest.mark.parametrize("name,sig", [("RX", "X"), ("RY", "Y"), ("RZ", "Z")])
@pytest.mark.parametrize("a", [0.0, 0.3, -1.7, np.pi, 7.85397, -3.0])
def test_rotation_is_matrix_exponential(name, sig, a):
    ref = sla.expm(-0.5j * a * PAULI_TEXTBOOK[sig])
    got = g.ONE_QUBIT_ROT[name](a)
    assert np.allclose(got, ref, atol=1e-14, rtol=0)


def test_fixed_gate_identities():
    assert np.allclose(g.H @ g.H, np.eye(2))
    assert np.allclose(g.S @ g.S, g.Z)
    assert np.allclose(g.T @ g.T, g.S)
    assert np.allclose(g.S @ g.SDG, np.eye(2))
    assert np.allclose(g.H @ g.X @ g.H, g.Z)
    assert np.allclose(g.rx(np.pi), -1j * g.X)
    assert np.allclose(g.ry(np.pi), -1j * g.Y)
    assert np.allclose(g.rz(np.pi), -1j * g.Z)
    assert np.allclose(g.X @ g.Y, 1j * g.Z)


def test_two_qubit_truth_tables():
    cnot = g.two_qubit("CNOT")
    # basis |control, target>, index 2*c + t
    for c in range(2):
        for t in range(2):
            e = np.zeros(4)
            e[2 * c + t] = 1
            out = cnot @ e
            assert out[2 * c + (t ^ c)] == 1
    assert np.allclose(g.two_qubit("CZ"), np.diag([1, 1, 1, -1]))
    sw = g.two_qubit("SWAP")
    assert np.allclose(sw @ sw, np.eye(4))
    assert sw[1, 2] == 1 and sw[2, 1] == 1
    # CZ = (I x H) CNOT (I x H)
    IH = np.kron(np.eye(2), g.H)
    assert np.allclose(IH @ cnot @ IH, g.two_qubit("CZ"))


def test_cnot_sandwich_is_zz_rotation():
    """CNOT(1->0) RZ_0(t) CNOT(1->0) = exp(-i t Z0 Z1 / 2): the identity that
    makes the paper's two-qubit VQE energy a + b cos t + c sin t."""
    # operator on qubits (0, 1) in basis 2*s0 + s1; CNOT with control 1 on 0
    sw = g.two_qubit("SWAP")
    cnot_10 = sw @ g.two_qubit("CNOT") @ sw
    for t in (0.0, 0.4, -2.2, np.pi):
        rz0 = np.kron(g.rz(t), np.eye(2))
        lhs = cnot_10 @ rz0 @ cnot_10
        rhs = sla.expm(-0.5j * t * np.kron(PAULI_TEXTBOOK["Z"], PAULI_TEXTBOOK["Z"]))
        assert np.allclose(lhs, rhs, atol=1e-14)
