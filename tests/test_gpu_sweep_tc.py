"""GPU parity of the tensor-core transfer sweeps (dtype c64_bf16split): the
BF16-split expectation values against the FP64 oracle, and against the FP32
(c64) sweeps on the very same states (the two forms share the state
simulation, so their difference is the split-precision sweep alone).

Bound used for the split products: every operand value is hi + lo to 2^-18
relative and each product drops lo*lo (2^-18), so one complex product carries
~3e-5 relative error at worst; a term's error relative to its scale stays
well inside 1e-4 for the sweep lengths used here."""
import numpy as np
import pytest

from oracle import energy as OE
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

SPLIT = "c64_bf16split"


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


def run(n, chi, eps, circ, thetas, terms, dtype, chunk=0):
    B = thetas.shape[0] if thetas is not None and np.ndim(thetas) == 2 else 1
    P = thetas.shape[-1] if thetas is not None else 0
    m = tnmps.MPSBatch(n, chi, B, dtype=dtype, max_params=P, eps=eps)
    m.apply_circuit(circ, thetas)
    ps = tnmps.PauliSum(n, terms)
    e, pt = m.expect(ps, per_term=True, chunk=chunk)
    m.check()
    return m, e, pt


def test_hea8_split_against_dense():
    wl = inputs.workload("hea8", 0)
    th = wl["thetas"]
    m, e, pt = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"], SPLIT)
    for b in range(th.shape[0]):
        ref = OE.term_values_dense(wl["n"], wl["circuit"], th[b], wl["terms"])
        assert np.max(np.abs(pt[b] - ref)) <= 1e-4
        assert abs(e[b] - OE.energy_from_values(wl["terms"], ref)) <= 1e-6 * sum_abs(wl["terms"])


def test_heis40_split_energy_target():
    """|dE| against the FP64 oracle MPS, the mixed form's stated target."""
    wl = inputs.workload("heis40")
    th = wl["thetas"][:4]
    m, e, pt = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"], SPLIT)
    _, e64, pt64 = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"], "c64")
    scale = sum_abs(wl["terms"])
    assert np.max(np.abs(pt - pt64)) <= 1e-4
    for b in range(2):
        vals, _ = OE.term_values_mps(wl["n"], wl["circuit"], th[b], wl["terms"], wl["chi_max"],
                                     wl["eps"])
        eref = OE.energy_from_values(wl["terms"], vals)
        assert abs(e[b] - eref) <= 1e-6 * scale, (e[b], eref, scale)


def test_random_strings_with_gaps_against_c64():
    """Weight <= 4 strings on 40 qubits (identity gaps inside the spans, all
    three Paulis, long spans) on chi = 64 states, per term against the FP32
    sweeps on the same states."""
    wl = inputs.workload("heis40")
    th = wl["thetas"][:3]
    terms = inputs.random_pauli_terms(40, 300, 4, np.random.default_rng(17), scale_by_weight=True)
    _, e, pt = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, terms, SPLIT, chunk=2)
    _, e64, pt64 = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, terms, "c64", chunk=2)
    assert np.all(np.abs(pt) <= 1 + 1e-4)
    assert np.max(np.abs(pt - pt64)) <= 1e-4
    assert np.max(np.abs(e - e64)) <= 1e-6 * sum_abs(terms)


def test_ragged_batch_product_and_entangled_states():
    """States of one batch with different bond dimensions: theta = 0 keeps the
    HEA state a product state (all bonds 1), random theta entangles it."""
    n, chi = 12, 32
    circ, P = inputs.hea_circuit(n, 3, ("RY", "RZ"))
    th = inputs.thetas(3, P, np.random.default_rng(3))
    th[1] = 0.0
    terms = inputs.random_pauli_terms(n, 60, 4, np.random.default_rng(4))
    m, e, pt = run(n, chi, 1e-12, circ, th, terms, SPLIT)
    dims = m.bond_dims()
    assert np.all(dims[1] == 1) and dims[0].max() > 1
    for b in range(3):
        ref = OE.term_values_dense(n, circ, th[b], terms)
        assert np.max(np.abs(pt[b] - ref)) <= 1e-4


def test_ghz40_long_strings():
    n = 40
    circ = [("H", 0, -1, -1, 0.0, 1.0)] + [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    terms = [(1.0, tuple(range(n)), (1,) * n), (1.0, tuple(range(n)), (2, 2) + (1,) * (n - 2)),
             (1.0, (3, 31), (3, 3)), (1.0, (17,), (3,)), (1.0, (0, 39), (3, 3))]
    m, e, pt = run(n, 8, 1e-10, circ, None, terms, SPLIT)
    assert np.allclose(pt[0], [1, -1, 1, 0, 1], atol=1e-4)


def test_chi128_saturated_states_against_oracle_and_c64():
    """Two states of the chi = 128 benchmark workload (middle bonds at 128)
    with 200 of its random strings and its Heisenberg chain: against the FP64
    oracle MPS on the same rows, and against the FP32 sweeps on the very same
    states (which isolates the split-precision sweep)."""
    wl = inputs.workload("chi128")
    th = wl["thetas"][:2]
    terms = wl["terms"] + wl["terms_random"][:200]
    m, e, pt = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, terms, SPLIT, chunk=1)
    assert m.bond_dims().max() == 128
    _, e64, pt64 = run(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, terms, "c64", chunk=1)
    assert np.max(np.abs(pt - pt64)) <= 1e-4
    assert np.max(np.abs(e - e64)) <= 1e-6 * sum_abs(terms)
    vals, om = OE.term_values_mps(wl["n"], wl["circuit"], th[0], terms, wl["chi_max"], wl["eps"])
    assert np.array(om.cut_margins)[:, 1].min() > 1e-5      # no tie at the chi_max cut
    assert np.max(np.abs(pt[0] - vals)) <= 1e-4
    assert abs(e[0] - OE.energy_from_values(terms, vals)) <= 1e-6 * sum_abs(terms)


def test_chi256_bonds_above_128_split_against_oracle():
    """Bonds up to the library's maximum (256): the tensor-core block
    contraction with several 128-wide N tiles and two row tiles, the sweeps'
    256-wide MMA variant and the 512-row Jacobi, against the FP64 oracle MPS
    (the cap binds at 256 in the middle) and against the FP32 forms."""
    n, chi = 18, 256
    circ, P = inputs.hea_circuit(n, 9, ("RY", "RZ"))
    th = inputs.thetas(2, P, np.random.default_rng(256))
    terms = inputs.heisenberg_terms(n, np.random.default_rng(257)) + \
        inputs.random_pauli_terms(n, 200, 4, np.random.default_rng(258), scale_by_weight=True)
    m, e, pt = run(n, chi, 1e-10, circ, th, terms, SPLIT)
    assert m.bond_dims().max() > 128
    m64, e64, pt64 = run(n, chi, 1e-10, circ, th, terms, "c64")
    # the two forms may cut a singular value at the threshold differently
    assert np.abs(m.bond_dims().astype(int) - m64.bond_dims()).max() <= 2
    assert np.max(np.abs(pt - pt64)) <= 1e-4
    assert np.max(np.abs(e - e64)) <= 1e-6 * sum_abs(terms)
    for b in range(2):
        vals, om = OE.term_values_mps(n, circ, th[b], terms, chi, 1e-10)
        assert max(om.bond_dims()) == chi
        assert np.array(om.cut_margins)[:, 1].min() > 1e-5
        assert np.max(np.abs(pt[b] - vals)) <= 1e-4
        assert abs(e[b] - OE.energy_from_values(terms, vals)) <= 1e-6 * sum_abs(terms)
