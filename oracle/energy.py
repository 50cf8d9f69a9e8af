"""Variational energy E(theta) = sum_k c_k <psi(theta)|P_k|psi(theta)> and its
parameter-shift gradient (oracle side; test infrastructure only).

Sec. V.B of the paper evaluates, for every parameter value, the expectation
of each Hamiltonian measurement term on the ansatz state; the energy is their
coefficient-weighted sum. The oracle evaluates each term exactly (no shot
sampling -- the paper does not specify shots), either on the dense state
vector (n <= 12) or on the FP64 MPS.

A Pauli sum is given as a list of terms ``(coeff, sites, paulis)`` with
Pauli codes 1=X, 2=Y, 3=Z.

Pins: the two-qubit closed form a + b cos t + c sin t of the paper's H2
ansatz (``tests/test_oracle_energy.py``), dense-vs-MPS agreement, the
two-site Heisenberg spectrum, and the parameter-shift rule against central
finite differences.
"""
import numpy as np

from . import mps as mps_mod
from . import statevector as sv


def term_values_dense(n, circuit, theta, terms):
    psi = sv.run_circuit(n, circuit, theta)
    return np.array([sv.pauli_expectation(psi, n, s, p).real for _, s, p in terms])


def term_values_mps(n, circuit, theta, terms, chi_max=1 << 30, eps=1e-4):
    m = mps_mod.MPS(n, chi_max=chi_max, eps=eps).run(circuit, theta)
    return np.array([m.expect_pauli(s, p).real for _, s, p in terms]), m


def energy_from_values(terms, values):
    # fixed term order, plain FP64 accumulation
    e = 0.0
    for (c, _, _), v in zip(terms, values):
        e += float(c) * float(v)
    return e


def energy(n, circuit, theta, terms, method="mps", chi_max=1 << 30, eps=1e-4):
    if method == "dense":
        vals = term_values_dense(n, circuit, theta, terms)
    else:
        vals, _ = term_values_mps(n, circuit, theta, terms, chi_max, eps)
    return energy_from_values(terms, vals)


def parameter_shift_gradient(n, circuit, theta, terms, method="mps", chi_max=1 << 30,
                             eps=1e-4):
    """dE/dtheta_j = [E(theta + pi/2 e_j) - E(theta - pi/2 e_j)] / 2, exact for
    gates exp(-i theta_j sigma / 2) with each parameter used once at scale 1."""
    used = {}
    for gate in circuit:
        p = gate[3]
        if p is not None and p >= 0:
            if float(gate[5]) != 1.0:
                raise ValueError("parameter-shift oracle needs unit scales")
            used[p] = used.get(p, 0) + 1
    if any(c != 1 for c in used.values()):
        raise ValueError("parameter-shift oracle needs each parameter used once")
    theta = np.asarray(theta, dtype=np.float64)
    grad = np.zeros_like(theta)
    for j in range(theta.size):
        if j not in used:
            continue
        tp, tm = theta.copy(), theta.copy()
        tp[j] += 0.5 * np.pi
        tm[j] -= 0.5 * np.pi
        grad[j] = 0.5 * (energy(n, circuit, tp, terms, method, chi_max, eps)
                         - energy(n, circuit, tm, terms, method, chi_max, eps))
    return grad
