"""Pins of the dense brute-force oracle: basis convention, Pauli expectations
against explicit Kronecker-product matrices, and closed forms."""
import functools

import numpy as np
import pytest

from oracle import gates as g
from oracle import statevector as sv

TEXTBOOK = {
    0: np.eye(2, dtype=complex),
    1: np.array([[0, 1], [1, 0]], dtype=complex),
    2: np.array([[0, -1j], [1j, 0]], dtype=complex),
    3: np.array([[1, 0], [0, -1]], dtype=complex),
}


def kron_string(n, sites, paulis):
    """Full 2^n matrix with qubit 0 as the least significant (rightmost)
    Kronecker factor."""
    ops = {q: p for q, p in zip(sites, paulis)}
    mats = [TEXTBOOK[ops.get(q, 0)] for q in range(n - 1, -1, -1)]
    return functools.reduce(np.kron, mats)


def test_basis_index_convention():
    n = 5
    for q in range(n):
        psi = sv.apply_1q(sv.zero_state(n), n, g.X, q)
        assert np.argmax(np.abs(psi)) == 1 << q


def test_cnot_direction_on_dense():
    n = 3
    psi = sv.apply_1q(sv.zero_state(n), n, g.X, 2)          # |100> : qubit 2 set
    psi = sv.apply_2q(psi, n, g.two_qubit("CNOT"), 2, 0)   # control 2, target 0
    assert np.argmax(np.abs(psi)) == 0b101


@pytest.mark.parametrize("seed", range(4))
def test_pauli_expectation_matches_kronecker(seed):
    rng = np.random.default_rng(seed)
    n = 5
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    for _ in range(20):
        w = int(rng.integers(0, n + 1))
        sites = list(rng.choice(n, size=w, replace=False))
        paulis = list(rng.integers(1, 4, size=w))
        ref = np.vdot(psi, kron_string(n, sites, paulis) @ psi)
        got = sv.pauli_expectation(psi, n, sites, paulis)
        assert abs(got - ref) < 1e-13


def test_product_state_bloch_closed_form():
    rng = np.random.default_rng(7)
    n = 6
    th = rng.uniform(-np.pi, np.pi, n)
    ph = rng.uniform(-np.pi, np.pi, n)
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    circ += [("RZ", q, -1, n + q, 0.0, 1.0) for q in range(n)]
    psi = sv.run_circuit(n, circ, np.concatenate([th, ph]))
    for q in range(n):
        assert abs(sv.pauli_expectation(psi, n, [q], [3]) - np.cos(th[q])) < 1e-13
        assert abs(sv.pauli_expectation(psi, n, [q], [1]) - np.sin(th[q]) * np.cos(ph[q])) < 1e-13
        assert abs(sv.pauli_expectation(psi, n, [q], [2]) - np.sin(th[q]) * np.sin(ph[q])) < 1e-13
    # strings factorise on a product state
    val = sv.pauli_expectation(psi, n, [0, 3, 5], [3, 1, 3])
    ref = np.cos(th[0]) * np.sin(th[3]) * np.cos(ph[3]) * np.cos(th[5])
    assert abs(val - ref) < 1e-13


def test_ghz_correlations():
    n = 7
    circ = [("H", 0, -1, -1, 0.0, 1.0)] + [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    psi = sv.run_circuit(n, circ, [])
    assert abs(sv.pauli_expectation(psi, n, list(range(n)), [1] * n) - 1) < 1e-13
    assert abs(sv.pauli_expectation(psi, n, [0, 4], [3, 3]) - 1) < 1e-13
    assert abs(sv.pauli_expectation(psi, n, [2], [3])) < 1e-13
    # Y Y X ... X on GHZ gives -1
    assert abs(sv.pauli_expectation(psi, n, list(range(n)), [2, 2] + [1] * (n - 2)) + 1) < 1e-13
