"""Pins of the energy oracle: the closed-form energy of the paper's two-qubit
VQE ansatz, the two-site Heisenberg spectrum, the parameter-shift rule against
finite differences, and dense-vs-MPS agreement."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import energy as E
from paper_1807_07914_gb300 import inputs

PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PI = np.eye(2, dtype=complex)
TB = {0: PI, 1: PX, 2: PY, 3: PZ}


def on0(U):   # qubit 0 is the least significant Kronecker factor
    return np.kron(PI, U)


def on1(U):
    return np.kron(U, PI)


def rot(sig, a):
    return sla.expm(-0.5j * a * sig)


def closed_form_coeffs(terms):
    """a, b, c of E(t) = a + b cos t + c sin t for the Sec. V.B ansatz, built
    from scipy matrix exponentials (independent of the oracle's gate code)."""
    V1 = on0(rot(PX, 7.85397)) @ on1(rot(PY, 1.57079)) @ on0(rot(PX, 3.1415926))
    V2 = on0(rot(PX, 1.57079)) @ on1(rot(PY, 7.8539752))
    phi = V1 @ np.array([1, 0, 0, 0], dtype=complex)
    Hm = np.zeros((4, 4), dtype=complex)
    for c, s, p in terms:
        ops = {q: pp for q, pp in zip(s, p)}
        Hm += c * np.kron(TB[ops.get(1, 0)], TB[ops.get(0, 0)])
    Hp = V2.conj().T @ Hm @ V2
    G = np.kron(PZ, PZ)
    ev = lambda A: np.vdot(phi, A @ phi)
    a = 0.5 * (ev(Hp) + ev(G @ Hp @ G))
    b = 0.5 * (ev(Hp) - ev(G @ Hp @ G))
    c = 0.5j * ev(G @ Hp - Hp @ G)
    for v in (a, b, c):
        assert abs(v.imag) < 1e-13
    return a.real, b.real, c.real


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("method", ["dense", "mps"])
def test_h2_ansatz_closed_form(seed, method):
    terms = inputs.all_two_qubit_terms(np.random.default_rng(seed))
    circ, _ = inputs.h2_ansatz()
    a, b, c = closed_form_coeffs(terms)
    scale = sum(abs(t[0]) for t in terms)
    for t in np.linspace(-np.pi, np.pi, 100):
        got = E.energy(2, circ, [t], terms, method=method, eps=1e-14)
        ref = a + b * np.cos(t) + c * np.sin(t)
        assert abs(got - ref) <= 1e-10 * scale


def test_heisenberg_two_site_spectrum():
    terms = [(1.0, (0, 1), (p, p)) for p in (1, 2, 3)]
    # H0, CNOT01, X1, Z0 prepares the singlet (energy -3); H0, CNOT01 a triplet (+1)
    singlet = [("H", 0, -1, -1, 0, 1), ("CNOT", 0, 1, -1, 0, 1), ("X", 1, -1, -1, 0, 1),
               ("Z", 0, -1, -1, 0, 1)]
    triplet = singlet[:2]
    for method in ("dense", "mps"):
        assert abs(E.energy(2, singlet, [], terms, method) + 3) < 1e-13
        assert abs(E.energy(2, triplet, [], terms, method) - 1) < 1e-13
    w = np.linalg.eigvalsh(sum(np.kron(TB[p], TB[p]) for p in (1, 2, 3)))
    assert np.allclose(sorted(w), [-3, 1, 1, 1])


def test_parameter_shift_matches_finite_difference():
    rng = np.random.default_rng(9)
    n = 4
    circ, P = inputs.hea_circuit(n, 2, ("RY", "RZ"))
    terms = inputs.random_pauli_terms(n, 10, 3, rng)
    th = rng.uniform(-np.pi, np.pi, P)
    grad = E.parameter_shift_gradient(n, circ, th, terms, method="dense")
    h = 1e-5
    for j in range(P):
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (E.energy(n, circ, tp, terms, "dense") - E.energy(n, circ, tm, terms, "dense")) / (2 * h)
        assert abs(fd - grad[j]) < 1e-7


def test_dense_and_mps_energies_agree_hea8():
    wl = inputs.workload("hea8")
    for b in range(4):
        th = wl["thetas"][b]
        ed = E.energy(8, wl["circuit"], th, wl["terms"], "dense")
        em = E.energy(8, wl["circuit"], th, wl["terms"], "mps", chi_max=16, eps=wl["eps"])
        assert abs(ed - em) < 1e-12
