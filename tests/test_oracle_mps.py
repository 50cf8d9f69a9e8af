"""Pins of the FP64 MPS oracle: exact agreement with the dense brute force when
nothing is truncated, unit norm after every gate, truncation error equal to
the discarded weight, closed forms at n=40, bond bounds, cutoff semantics."""
import numpy as np
import pytest

from oracle import gates as g
from oracle import mps as M
from oracle import statevector as sv
from paper_1807_07914_gb300 import inputs


def run_both(n, circ, theta, chi=1 << 20, eps=1e-14):
    m = M.MPS(n, chi_max=chi, eps=eps).run(circ, theta)
    return m, sv.run_circuit(n, circ, theta)


@pytest.mark.parametrize("rep", range(3))
def test_hea8_matches_dense_per_term(rep):
    wl = inputs.workload("hea8", rep)
    for b in range(3):
        th = wl["thetas"][b]
        m = M.MPS(wl["n"], chi_max=wl["chi_max"], eps=wl["eps"]).run(wl["circuit"], th)
        psi = sv.run_circuit(wl["n"], wl["circuit"], th)
        assert m.discarded < 1e-24
        for _, s, p in wl["terms"]:
            assert abs(m.expect_pauli(s, p) - sv.pauli_expectation(psi, wl["n"], s, p)) < 1e-12
        # the whole state agrees too
        assert np.allclose(m.to_dense(), psi, atol=1e-12)


def test_norm_is_one_after_every_gate():
    rng = np.random.default_rng(3)
    circ, P = inputs.hea_circuit(9, 3, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, P)
    m = M.MPS(9, chi_max=64, eps=1e-12)
    for gate in circ:
        m.run([gate], th)
        assert abs(m.norm2() - 1.0) < 1e-12


@pytest.mark.parametrize("chi", [1, 2, 3])
def test_truncation_error_equals_discarded_weight(chi):
    rng = np.random.default_rng(11 + chi)
    n = 8
    circ, P = inputs.hea_circuit(n, 3, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, P)
    m = M.MPS(n, chi_max=64, eps=1e-14).run(circ, th)
    psi = m.to_dense()
    # one more entangler across the middle with a small cap
    G = g.two_qubit("CNOT") @ np.kron(g.ry(0.7), g.rx(-1.1))
    exact = sv.apply_2q(psi, n, G, 3, 4)
    m.chi_max = chi
    m.apply_2q(G, 3, 4)
    w = m.step_weights[-1]
    assert w > 1e-6
    kept = m.to_dense() * np.sqrt(1.0 - w)
    err = np.linalg.norm(exact - kept) ** 2
    assert abs(err - w) <= 1e-10 * w
    assert abs(m.norm2() - 1.0) < 1e-12


def test_non_adjacent_and_reversed_gates_match_dense():
    rng = np.random.default_rng(5)
    n = 7
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    circ += [("CNOT", 0, 5, -1, 0.0, 1.0), ("CZ", 6, 2, -1, 0.0, 1.0),
             ("CNOT", 4, 3, -1, 0.0, 1.0), ("SWAP", 1, 6, -1, 0.0, 1.0),
             ("RX", 3, -1, n, 0.0, 1.0), ("CNOT", 6, 0, -1, 0.0, 1.0)]
    th = rng.uniform(-np.pi, np.pi, n + 1)
    m, psi = run_both(n, circ, th)
    assert np.allclose(m.to_dense(), psi, atol=1e-12)


def test_ghz_n40_closed_form():
    n = 40
    circ = [("H", 0, -1, -1, 0.0, 1.0)] + [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    m = M.MPS(n, chi_max=64, eps=1e-10).run(circ, [])
    assert m.bond_dims() == [2] * (n - 1)
    assert abs(m.expect_pauli(list(range(n)), [1] * n) - 1) < 1e-12
    assert abs(m.expect_pauli(list(range(n)), [2, 2] + [1] * (n - 2)) + 1) < 1e-12
    assert abs(m.expect_pauli([3, 31], [3, 3]) - 1) < 1e-12
    assert abs(m.expect_pauli([17], [3])) < 1e-12


def test_product_state_n40_closed_form():
    rng = np.random.default_rng(2)
    n = 40
    th = rng.uniform(-np.pi, np.pi, 2 * n)
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    circ += [("RZ", q, -1, n + q, 0.0, 1.0) for q in range(n)]
    m = M.MPS(n).run(circ, th)
    bloch = lambda q, p: (np.sin(th[q]) * np.cos(th[n + q]), np.sin(th[q]) * np.sin(th[n + q]),
                          np.cos(th[q]))[p - 1]
    for _ in range(10):
        w = int(rng.integers(1, 5))
        s = sorted(rng.choice(n, size=w, replace=False))
        p = list(rng.integers(1, 4, size=w))
        ref = np.prod([bloch(q, pp) for q, pp in zip(s, p)])
        assert abs(m.expect_pauli(s, p) - ref) < 1e-12


@pytest.mark.parametrize("layers", [1, 2, 3, 4])
def test_bond_dimension_bounds(layers):
    rng = np.random.default_rng(layers)
    n = 12
    circ, P = inputs.hea_circuit(n, layers, ("RY", "RZ"))
    m = M.MPS(n, chi_max=1 << 20, eps=1e-12).run(circ, rng.uniform(-np.pi, np.pi, P))
    for i, d in enumerate(m.bond_dims()):
        assert d <= min(2 ** layers, 2 ** (i + 1), 2 ** (n - i - 1))


@pytest.mark.parametrize("s,expected_dim", [(5e-5, 1), (2e-4, 2)])
def test_cutoff_is_relative_on_singular_values(s, expected_dim):
    """cos(a)|00> + sin(a)|11> has Schmidt values (cos a, sin a); the paper's
    default cutoff 1e-4 drops sin a = 5e-5 and keeps 2e-4."""
    a = np.arcsin(s)
    circ = [("RY", 0, -1, -1, 2 * a, 1.0), ("CNOT", 0, 1, -1, 0.0, 1.0)]
    m = M.MPS(2, chi_max=8, eps=1e-4).run(circ, [])
    assert m.bond_dims() == [expected_dim]
    if expected_dim == 1:
        assert abs(m.discarded - s * s) < 1e-18
        assert abs(m.expect_pauli([0], [3]) - 1.0) < 1e-12


def test_cut_margin_closed_forms():
    """The truncation-decision margins: distance of sigma from the relative
    cutoff, and the gap at the chi_max cut when the cap binds (both relative
    to sigma_0)."""
    a = np.arcsin(5e-5)
    d_cut, d_cap = M.cut_margin([np.cos(a), np.sin(a)], 8, 1e-4)
    assert abs(d_cut - 5e-5 / np.cos(a)) < 1e-15 and d_cap == np.inf
    s = [0.8, 0.4, 0.4 - 1e-9, 0.1]
    d_cut, d_cap = M.cut_margin(s, 2, 1e-10)                          # cap binds: the gap
    assert abs(d_cap - 1e-9 / 0.8) < 1e-15
    assert abs(d_cut - (0.1 - 1e-10 * np.linalg.norm(s)) / 0.8) < 1e-15
    assert M.cut_margin(s, 4, 1e-10)[1] == np.inf
    # a Bell pair cut to one value: equal Schmidt values, an exact tie
    circ = [("H", 0, -1, -1, 0.0, 1.0), ("CNOT", 0, 1, -1, 0.0, 1.0)]
    m = M.MPS(2, chi_max=1, eps=1e-10).run(circ, [])
    assert m.cut_margins[-1][1] < 1e-15 and abs(m.discarded - 0.5) < 1e-15
    m = M.MPS(2, chi_max=2, eps=1e-10).run(circ, [])
    assert abs(m.cut_margins[-1][0] - (1 - np.sqrt(2) * 1e-10)) < 1e-14
    assert m.cut_margins[-1][1] == np.inf


def test_rounds_circuit_two_rounds_bond_four():
    """Sec. V.A: after two random rounds the maximum bond dimension is 4,
    independent of the register size."""
    rng = np.random.default_rng(0)
    for n in (5, 10, 25):
        circ = inputs.rounds_circuit(n, 2, rng)
        m = M.MPS(n, chi_max=1 << 10, eps=1e-12).run(circ, [])
        assert max(m.bond_dims()) <= 4
