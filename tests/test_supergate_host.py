"""The library's host-side super-gate builder (CPU, no GPU): its MPO equals
the product of the gate matrices, and its bonds are the exact ranks of the
operator's cuts."""
import numpy as np
import pytest

from oracle import gates as G
from oracle import statevector as SV

BLOCK = [("CNOT", 2, 5, -1, 0.0, 1.0), ("RY", 3, -1, 0, 0.0, 1.0), ("CZ", 6, 3, -1, 0.0, 1.0),
         ("SWAP", 4, 2, -1, 0.0, 1.0), ("H", 5, -1, -1, 0.0, 1.0), ("RZ", 1, -1, 1, 0.0, 1.0),
         ("CNOT", 6, 1, -1, 0.0, 1.0), ("RX", 4, -1, -1, 0.7, 1.0), ("CNOT", 1, 2, -1, 0.0, 1.0)]
THETA = np.array([0.9, -1.3])


@pytest.fixture(scope="module")
def T():
    from paper_1807_07914_gb300 import build, tnmps
    build.build()
    return tnmps


def dense_block(circuit, theta, p, m):
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


def contract(W):
    """MPO -> dense matrix with bit i = window site i."""
    T = W[0][0]
    m = 1
    for Wi in W[1:]:
        T = np.einsum("xyb,bosc->xoysc", T, Wi)
        m += 1
        T = T.reshape(2 ** m, 2 ** m, -1)
    T = T[:, :, 0].reshape((2,) * (2 * m))
    perm = tuple(range(m - 1, -1, -1)) + tuple(range(2 * m - 1, m - 1, -1))
    return T.transpose(perm).reshape(2 ** m, 2 ** m)


def cut_ranks(D, m):
    """Rank of the operator split after each window site."""
    t = D.reshape((2,) * (2 * m))
    # axes of t: out bits m-1..0 then in bits m-1..0; to site order
    t = t.transpose(tuple(range(m - 1, -1, -1)) + tuple(range(2 * m - 1, m - 1, -1)))
    ranks = []
    for k in range(1, m):
        left = list(range(k)) + [m + i for i in range(k)]
        right = [i for i in range(m) if i >= k] + [m + i for i in range(m) if i >= k]
        M = t.transpose(left + right).reshape(4 ** k, -1)
        s = np.linalg.svd(M, compute_uv=False)
        ranks.append(int(np.count_nonzero(s > 1e-10 * s[0])))
    return ranks


@pytest.mark.parametrize("circuit,theta", [
    (BLOCK, THETA),
    ([("CNOT", 5, 4, -1, 0.0, 1.0)], None),
    ([("SWAP", 0, 3, -1, 0.0, 1.0), ("RY", 1, -1, 0, 0.0, 1.0), ("CZ", 3, 1, -1, 0.0, 1.0)],
     np.array([0.4])),
    ([("CNOT", 0, 6, -1, 0.0, 1.0), ("CNOT", 6, 0, -1, 0.0, 1.0), ("CNOT", 0, 6, -1, 0.0, 1.0)],
     None),
])
def test_mpo_equals_gate_product_with_minimal_bonds(T, circuit, theta):
    sg = T.Supergate(10, circuit, theta)
    qs = [g[1] for g in circuit] + [g[2] for g in circuit if G.is_two_qubit(g)]
    assert (sg.first, sg.last) == (min(qs), max(qs))
    m = sg.last - sg.first + 1
    W = sg.mpo()
    D = dense_block(circuit, theta, sg.first, m)
    np.testing.assert_allclose(contract(W), D, atol=1e-12)
    assert list(sg.bonds[1:-1]) == cut_ranks(D, m)
    assert sg.bonds[0] == 1 and sg.bonds[-1] == 1
    sg.close()


def test_three_cnots_make_a_swap_of_rank_four(T):
    # CNOT(a,b) CNOT(b,a) CNOT(a,b) = SWAP(a,b): rank 4 across every cut
    sg = T.Supergate(8, [("CNOT", 1, 4, -1, 0.0, 1.0), ("CNOT", 4, 1, -1, 0.0, 1.0),
                         ("CNOT", 1, 4, -1, 0.0, 1.0)])
    assert list(sg.bonds) == [1, 4, 4, 4, 1]


def test_bad_gates_rejected(T):
    with pytest.raises(T.TnmpsError):
        T.Supergate(4, [("CNOT", 1, 4, -1, 0.0, 1.0)])        # qubit out of range
    with pytest.raises(T.TnmpsError):
        T.Supergate(4, [("RY", 1, -1, 2, 0.0, 1.0)], np.zeros(2))  # parameter index
    with pytest.raises(T.TnmpsError):
        T.Supergate(4, [("CZ", 2, 2, -1, 0.0, 1.0)])          # same qubit twice


def test_empty_and_one_qubit_super_gates(T):
    with pytest.raises(T.TnmpsError):
        T.Supergate(4, [])
    sg = T.Supergate(6, [("RY", 3, -1, 0, 0.0, 1.0), ("H", 3, -1, -1, 0.0, 1.0)], np.array([0.4]))
    assert (sg.first, sg.last) == (3, 3) and list(sg.bonds) == [1, 1]
    W = sg.mpo()
    U = G.H @ G.ry(0.4)
    np.testing.assert_allclose(W[0][0, :, :, 0], U, atol=1e-14)
