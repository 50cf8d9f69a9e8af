"""Textbook gate matrices in complex128 (oracle side; test infrastructure only).

Conventions (readings of the paper, which is silent on them; Sec. V.B listing):

* Rotations are R_sigma(a) = exp(-i a sigma / 2) for sigma in {X, Y, Z}.
* ``CNOT c t``: first operand is the control, second the target (the listing
  writes "CNOT 1 0").
* A two-qubit matrix ``G`` acting on an ordered qubit pair (qa, qb) is written
  in the basis index ``2*s_a + s_b`` (qa is the more significant factor).

Pins: ``tests/test_oracle_gates.py`` checks every rotation against
``scipy.linalg.expm`` and the fixed gates against their defining identities
(H^2 = I, S^2 = Z, RX(pi) = -iX, CNOT truth table, ...).
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
SDG = np.array([[1, 0], [0, -1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(0.25j * np.pi)]], dtype=np.complex128)

PAULI = {0: I2, 1: X, 2: Y, 3: Z}


def rx(a):
    c, s = np.cos(a / 2.0), np.sin(a / 2.0)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(a):
    c, s = np.cos(a / 2.0), np.sin(a / 2.0)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(a):
    return np.array([[np.exp(-0.5j * a), 0], [0, np.exp(0.5j * a)]], dtype=np.complex128)


ONE_QUBIT_FIXED = {"I": I2, "X": X, "Y": Y, "Z": Z, "H": H, "S": S, "SDG": SDG, "T": T}
ONE_QUBIT_ROT = {"RX": rx, "RY": ry, "RZ": rz}
TWO_QUBIT = ("CNOT", "CZ", "SWAP")


def two_qubit(name):
    """4x4 matrix of a two-qubit gate on the ordered pair (first, second)
    operand, basis index 2*s_first + s_second."""
    m = np.zeros((4, 4), dtype=np.complex128)
    for sa in range(2):
        for sb in range(2):
            col = 2 * sa + sb
            if name == "CNOT":      # first = control, second = target
                ta, tb, ph = sa, sb ^ sa, 1.0
            elif name == "CZ":
                ta, tb, ph = sa, sb, (-1.0 if (sa and sb) else 1.0)
            elif name == "SWAP":
                ta, tb, ph = sb, sa, 1.0
            else:
                raise ValueError(f"unknown two-qubit gate {name}")
            m[2 * ta + tb, col] = ph
    return m


def gate_angle(gate, theta):
    """Effective rotation angle of a gate record (name, q0, q1, param, angle,
    scale): angle + scale * theta[param] when param >= 0, else angle."""
    name, q0, q1, param, angle, scale = gate
    if param is None or param < 0:
        return float(angle)
    return float(angle) + float(scale) * float(theta[param])


def one_qubit_matrix(gate, theta):
    name = gate[0]
    if name in ONE_QUBIT_FIXED:
        return ONE_QUBIT_FIXED[name]
    if name in ONE_QUBIT_ROT:
        return ONE_QUBIT_ROT[name](gate_angle(gate, theta))
    raise ValueError(f"not a one-qubit gate: {name}")


def is_two_qubit(gate):
    return gate[0] in TWO_QUBIT
