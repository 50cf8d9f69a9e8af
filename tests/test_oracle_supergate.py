"""Pins of the oracle's super-gate application by overlap maximisation (CPU)."""
import copy

import numpy as np
import pytest

from oracle import gates as G
from oracle import mps as OM
from oracle import statevector as SV
from oracle import supergate as SG
from oracle.mps import truncation_rank
from paper_1807_07914_gb300 import inputs

# a super-gate on qubits 1..6 with distant and reversed two-qubit gates
BLOCK = [("CNOT", 2, 5, -1, 0.0, 1.0), ("RY", 3, -1, 0, 0.0, 1.0), ("CZ", 6, 3, -1, 0.0, 1.0),
         ("SWAP", 4, 2, -1, 0.0, 1.0), ("H", 5, -1, -1, 0.0, 1.0), ("RZ", 1, -1, 1, 0.0, 1.0),
         ("CNOT", 6, 1, -1, 0.0, 1.0), ("RX", 4, -1, -1, 0.7, 1.0), ("CNOT", 1, 2, -1, 0.0, 1.0)]
BLOCK_THETA = np.array([0.9, -1.3])


def dense_block(circuit, theta, p, m):
    """The gate list as a 2^m x 2^m matrix on qubits p..p+m-1 (bit 0 = qubit
    p), column by column through the state-vector module."""
    D = np.zeros((1 << m, 1 << m), dtype=np.complex128)
    for k in range(1 << m):
        v = np.zeros(1 << m, dtype=np.complex128)
        v[k] = 1.0
        for gate in circuit:
            if G.is_two_qubit(gate):
                v = SV.apply_2q(v, m, G.two_qubit(gate[0]), gate[1] - p, gate[2] - p)
            else:
                v = SV.apply_1q(v, m, G.one_qubit_matrix(gate, theta), gate[1] - p)
        D[:, k] = v
    return D


def apply_dense(psi, n, circuit, theta):
    for gate in circuit:
        if G.is_two_qubit(gate):
            psi = SV.apply_2q(psi, n, G.two_qubit(gate[0]), gate[1], gate[2])
        else:
            psi = SV.apply_1q(psi, n, G.one_qubit_matrix(gate, theta), gate[1])
    return psi


def hea_state(n, layers, chi, seed, eps=1e-14):
    rng = np.random.default_rng(seed)
    circ, P = inputs.hea_circuit(n, layers, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, P)
    return OM.MPS(n, chi, eps).run(circ, th), SV.run_circuit(n, circ, th)


@pytest.mark.parametrize("circuit", [
    BLOCK,
    [("CNOT", 5, 4, -1, 0.0, 1.0)],
    [("SWAP", 0, 3, -1, 0.0, 1.0), ("RY", 1, -1, 0, 0.0, 1.0), ("CZ", 3, 1, -1, 0.0, 1.0)],
])
def test_mpo_equals_gate_product(circuit):
    p, q, W = SG.mpo_from_gates(circuit, BLOCK_THETA)
    assert (p, q) == SG.window(circuit)
    assert W[0].shape[0] == 1 and W[-1].shape[3] == 1
    ref = dense_block(circuit, BLOCK_THETA, p, q - p + 1)
    np.testing.assert_allclose(SG.mpo_dense(W), ref, atol=1e-13)


def test_schmidt_ranks_of_fixed_gates():
    # operator-Schmidt rank: CNOT and CZ 2, SWAP 4 (bond between the qubits)
    for name, r in (("CNOT", 2), ("CZ", 2), ("SWAP", 4)):
        _, _, W = SG.mpo_from_gates([(name, 0, 1, -1, 0.0, 1.0)], None)
        assert W[0].shape[3] == r


def test_exact_without_truncation():
    n = 8
    psi, dense = hea_state(n, 2, 64, 3)
    phi, F, hist, chi, _ = SG.apply_supergate(psi, BLOCK, BLOCK_THETA, chi_max=64, target=1e-12)
    ref = apply_dense(dense, n, BLOCK, BLOCK_THETA)
    assert abs(F - 1.0) < 1e-12
    np.testing.assert_allclose(phi.to_dense(), ref, atol=1e-10)
    # step (6) raised the cap from the copy's bonds until the fit was exact
    assert chi > max(psi.bond_dims()[1:6])
    # the sites outside the window are the input's
    ps = copy.deepcopy(psi)
    ps.move_centre(1)
    np.testing.assert_array_equal(phi.tensors[0], ps.tensors[0])
    np.testing.assert_array_equal(phi.tensors[7], ps.tensors[7])


def test_distant_cnot_closed_form():
    n = 6
    plus = OM.MPS(n, 8, 1e-14)
    plus.apply_1q(G.H, 0)
    cnot = [("CNOT", 0, 4, -1, 0.0, 1.0)]
    # best product-state approximation of (|0..0> + |1...1_4>)/sqrt(2): F = 1/2
    _, F1, _, chi1, _ = SG.apply_supergate(plus, cnot, None, chi_max=1)
    assert abs(F1 - 0.5) < 1e-12 and chi1 == 1
    phi, F2, _, chi2, _ = SG.apply_supergate(plus, cnot, None, chi_max=4)
    assert abs(F2 - 1.0) < 1e-12 and chi2 == 2
    assert phi.bond_dims() == [2, 2, 2, 2, 1]


def test_single_adjacent_gate_is_eckart_young():
    n = 6
    psi, _ = hea_state(n, 3, 8, 5)
    gates = [("RY", 2, -1, 0, 0.0, 1.0), ("CNOT", 2, 3, -1, 0.0, 1.0), ("RX", 3, -1, 1, 0.0, 1.0)]
    th = np.array([0.4, 1.1])
    ref = copy.deepcopy(psi)
    ref.chi_max = 2
    ref.run(gates, th)
    w = ref.step_weights[-1]
    assert w > 1e-3  # the cap truncates
    phi, F, hist, _, F0 = SG.apply_supergate(psi, gates, th, chi_max=2)
    assert abs(F - (1.0 - w)) < 1e-12 and abs(F0 - (1.0 - w)) < 1e-12
    np.testing.assert_allclose(phi.to_dense(), ref.to_dense(), atol=1e-10)


def test_sweeps_never_lower_the_first_iterate():
    n = 8
    psi, _ = hea_state(n, 3, 16, 7)
    phi, F, hist, chi, F0 = SG.apply_supergate(psi, BLOCK, BLOCK_THETA, chi_max=4, max_sweeps=6)
    assert chi == 4
    assert F >= F0 - 1e-12
    assert all(b >= a - 1e-12 for a, b in zip(hist, hist[1:]))
    assert F > F0 + 1e-4  # the sweeps beat gate-by-gate truncation here
    assert abs(phi.norm2() - 1.0) < 1e-12
    assert max(phi.bond_dims()) <= 4


def _dense_sweep(phi, target, p, q, chi):
    """The same left-to-right two-site updates, with the gradient taken from
    the dense target vector instead of MPO environments."""
    n = phi.n
    T = target.reshape((2,) * n).transpose(tuple(range(n - 1, -1, -1)))  # axis i = site i
    phi.move_centre(p)
    for i in range(p, q):
        Lm = np.ones((1, 1), dtype=np.complex128)
        for A in phi.tensors[:i]:
            Lm = np.einsum("xa,asb->xsb", Lm, A).reshape(-1, A.shape[2])
        Rm = np.ones((1, 1), dtype=np.complex128)
        for A in reversed(phi.tensors[i + 2:]):
            Rm = np.einsum("asb,by->asy", A, Rm).reshape(A.shape[0], -1)
        Tm = T.reshape(Lm.shape[0], 4, Rm.shape[1])
        grad = np.einsum("xa,xuy,cy->auc", Lm.conj(), Tm, Rm.conj())
        Fa, Fc = grad.shape[0], grad.shape[2]
        U, S, Vh = np.linalg.svd(grad.reshape(Fa, 2, 2, Fc).reshape(2 * Fa, 2 * Fc),
                                 full_matrices=False)
        k, _, kept = truncation_rank(S, chi, phi.eps)
        phi.tensors[i] = U[:, :k].reshape(Fa, 2, k)
        phi.tensors[i + 1] = ((S[:k, None] / kept) * Vh[:k]).reshape(k, 2, Fc)
        phi.centre = i + 1
    return abs(np.vdot(phi.to_dense(), target)) ** 2


def test_environments_match_dense_gradient():
    n = 8
    psi, dense = hea_state(n, 3, 16, 11)
    target = apply_dense(dense, n, BLOCK, BLOCK_THETA)
    p, q, W = SG.mpo_from_gates(BLOCK, BLOCK_THETA)
    ps = copy.deepcopy(psi)
    ps.move_centre(p)
    start = copy.deepcopy(ps)
    start.chi_max = 4
    start.run(BLOCK, BLOCK_THETA)
    a, b = copy.deepcopy(start), copy.deepcopy(start)
    f0 = SG.overlap_fidelity(a, ps, p, q, W)
    assert abs(f0 - abs(np.vdot(a.to_dense(), target)) ** 2) < 1e-12
    for _ in range(3):
        fa = SG.sweep(a, ps, p, q, W, 4)
        fb = _dense_sweep(b, target, p, q, 4)
        assert abs(fa - fb) < 1e-11
    np.testing.assert_allclose(abs(np.vdot(a.to_dense(), b.to_dense())), 1.0, atol=1e-10)


def test_one_qubit_window_is_exact():
    psi, dense = hea_state(5, 2, 8, 13)
    gates = [("RY", 2, -1, 0, 0.0, 1.0), ("H", 2, -1, -1, 0.0, 1.0)]
    phi, F, _, _, _ = SG.apply_supergate(psi, gates, np.array([0.3]), chi_max=8)
    assert F == 1.0
    np.testing.assert_allclose(phi.to_dense(), apply_dense(dense, 5, gates, np.array([0.3])),
                               atol=1e-12)
