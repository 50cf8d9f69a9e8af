"""Pins of the oracle's shot sampler (CPU)."""
import numpy as np
import pytest

from oracle import gates as G
from oracle import mps as OM
from oracle import sampling as S
from oracle import statevector as SV
from paper_1807_07914_gb300 import inputs


@pytest.mark.parametrize("n,layers", [(5, 2), (7, 3), (9, 2)])
def test_mps_and_dense_samplers_agree(n, layers):
    rng = np.random.default_rng(10 * n + layers)
    circ, P = inputs.hea_circuit(n, layers, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, P)
    psi = SV.run_circuit(n, circ, th)
    m = OM.MPS(n, 1 << 10, 1e-14).run(circ, th)
    u = rng.random((300, n))
    bd, md = S.sample_dense(psi, n, u)
    bm, mm = S.sample_mps(m, u)
    ok = np.minimum(md, mm) > 1e-9
    assert ok.mean() > 0.99
    assert np.array_equal(bd[ok], bm[ok])


def test_born_rule_histogram():
    n = 4
    rng = np.random.default_rng(3)
    circ, P = inputs.hea_circuit(n, 2, ("RY", "RZ"))
    psi = SV.run_circuit(n, circ, rng.uniform(-np.pi, np.pi, P))
    bits, _ = S.sample_dense(psi, n, rng.random((20000, n)))
    idx = (bits.astype(np.int64) << np.arange(n)).sum(axis=1)  # qubit q = bit q
    freq = np.bincount(idx, minlength=1 << n) / len(idx)
    assert 0.5 * np.abs(freq - np.abs(psi) ** 2).sum() < 0.02


@pytest.mark.parametrize("n", [7, 30])
def test_ghz_all_equal(n):
    m = OM.MPS(n, 4, 1e-12)
    m.apply_1q(G.one_qubit_matrix(("H", 0, -1, -1, 0.0, 1.0), None), 0)
    for q in range(n - 1):
        m.apply_2q(G.two_qubit("CNOT"), q, q + 1)
    u = np.random.default_rng(n).random((200, n))
    bits, _ = S.sample_mps(m, u)
    expect = (u[:, n - 1] >= 0.5).astype(np.uint8)   # the first draw decides
    assert np.array_equal(bits, np.repeat(expect[:, None], n, axis=1))
    if n <= 10:
        bd, _ = S.sample_dense(m.to_dense(), n, u)
        assert np.array_equal(bd, bits)


def test_product_state_closed_form():
    n = 20
    rng = np.random.default_rng(11)
    th = rng.uniform(-np.pi, np.pi, n)
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    m = OM.MPS(n, 4, 1e-12).run(circ, th)
    u = rng.random((500, n))
    bits, _ = S.sample_mps(m, u)
    assert np.array_equal(bits, (u >= np.cos(th / 2) ** 2).astype(np.uint8))
