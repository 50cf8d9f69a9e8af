"""Dense state-vector brute force (oracle side; test infrastructure only).

This is the exact, exponential-memory simulation that Sec. I of the paper
contrasts with tensor-network factorisations. It is used here only as the
ground truth for small registers (n <= 12).

Convention: qubit q is bit q of the basis-state index (qubit 0 is the least
significant bit); MPS site q holds qubit q.

Pins: ``tests/test_oracle_statevector.py`` -- basis-index convention, Pauli
expectations against explicit Kronecker-product matrices (brute force), the
product-state closed forms <Z>=cos, <X>=sin, and GHZ correlations.
"""
import numpy as np

from . import gates as g

MAX_QUBITS = 12


def zero_state(n):
    if not 1 <= n <= MAX_QUBITS:
        raise ValueError(f"dense oracle supports 1..{MAX_QUBITS} qubits, got {n}")
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def _axis(n, q):
    # numpy C-order reshape to (2,)*n puts bit n-1 on axis 0.
    return n - 1 - q


def apply_1q(psi, n, U, q):
    t = psi.reshape((2,) * n)
    ax = _axis(n, q)
    t = np.tensordot(U, t, axes=([1], [ax]))
    t = np.moveaxis(t, 0, ax)
    return t.reshape(-1)


def apply_2q(psi, n, G, qa, qb):
    """Apply a 4x4 G written in basis 2*s_qa + s_qb to qubits (qa, qb)."""
    if qa == qb:
        raise ValueError("two-qubit gate on a single qubit")
    t = psi.reshape((2,) * n)
    axa, axb = _axis(n, qa), _axis(n, qb)
    G4 = G.reshape(2, 2, 2, 2)  # [ta, tb, sa, sb]
    t = np.tensordot(G4, t, axes=([2, 3], [axa, axb]))
    t = np.moveaxis(t, [0, 1], [axa, axb])
    return t.reshape(-1)


def run_circuit(n, circuit, theta):
    """Return U(theta)|0...0> for a gate list of records
    (name, q0, q1, param, angle, scale)."""
    psi = zero_state(n)
    for gate in circuit:
        if g.is_two_qubit(gate):
            psi = apply_2q(psi, n, g.two_qubit(gate[0]), gate[1], gate[2])
        else:
            psi = apply_1q(psi, n, g.one_qubit_matrix(gate, theta), gate[1])
    return psi


def pauli_expectation(psi, n, sites, paulis):
    """<psi| P |psi> for the Pauli string P = prod_j sigma_{paulis[j]}(sites[j])
    (1=X, 2=Y, 3=Z), by bit-flip and phase indexing of the dense vector."""
    idx = np.arange(1 << n, dtype=np.int64)
    flip = 0
    phase = np.ones(1 << n, dtype=np.complex128)
    for q, p in zip(sites, paulis):
        bit = (idx >> q) & 1
        if p == 1:          # X|b> = |1-b>
            flip |= 1 << q
        elif p == 2:        # Y|0> = i|1>, Y|1> = -i|0>
            flip |= 1 << q
            phase *= np.where(bit == 0, 1j, -1j)
        elif p == 3:        # Z|b> = (-1)^b |b>
            phase *= np.where(bit == 0, 1.0, -1.0)
        else:
            raise ValueError(f"bad Pauli code {p}")
    # P|x> = phase(x) |x ^ flip>  =>  <psi|P|psi> = sum_x conj(psi[x^flip]) phase(x) psi[x]
    return complex(np.sum(np.conj(psi[idx ^ flip]) * phase * psi))
