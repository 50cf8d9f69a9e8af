"""GPU parity on the remaining workload shapes: the 100-qubit single state
(chi_max 256, cutoff 1e-8, 5000 strings) against the FP64 oracle on a 20-term
subset, and the random "rounds" circuits of Sec. V.A (H, Pauli and rotation
layers with CNOT ladders) against the dense oracle."""
import numpy as np
import pytest

from oracle import energy as OE
from oracle import mps as OM
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_bf16split"])
def test_large100_twenty_term_subset(dtype):
    wl = inputs.workload("large100")
    th = wl["thetas"][:1]
    sub = wl["terms"][:20]
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], 1, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.apply_circuit(wl["circuit"], th)
    e, pt = m.expect(tnmps.PauliSum(wl["n"], sub), per_term=True)
    m.check()
    vals, om = OE.term_values_mps(wl["n"], wl["circuit"], th[0], sub, wl["chi_max"], wl["eps"])
    scale = sum(abs(t[0]) for t in sub)
    eref = OE.energy_from_values(sub, vals)
    # six ladder layers: bonds <= 2^6, the chi cap never binds
    assert m.bond_dims().max() <= 64
    if dtype == "c128":
        assert list(m.bond_dims()[0]) == om.bond_dims()
        assert np.max(np.abs(pt[0] - vals)) <= 1e-10
    else:
        assert np.max(np.abs(pt[0] - vals)) <= 1e-4
        assert abs(e[0] - eref) <= 1e-6 * scale


def test_large100_all_terms_split_against_c64():
    """All 5000 strings on the 100-qubit state: the tensor-core sweeps against
    the FP32 sweeps on the same state."""
    wl = inputs.workload("large100")
    th = wl["thetas"][:1]
    out = {}
    for dtype in ("c64", "c64_bf16split"):
        m = tnmps.MPSBatch(wl["n"], wl["chi_max"], 1, dtype=dtype, max_params=wl["n_params"],
                           eps=wl["eps"])
        m.apply_circuit(wl["circuit"], th)
        out[dtype] = m.expect(tnmps.PauliSum(wl["n"], wl["terms"]), per_term=True)
        m.check()
    assert np.max(np.abs(out["c64"][1] - out["c64_bf16split"][1])) <= 1e-4
    scale = sum(abs(t[0]) for t in wl["terms"])
    assert abs(out["c64"][0][0] - out["c64_bf16split"][0][0]) <= 1e-6 * scale


@pytest.mark.parametrize("dtype", ["c128", "c64_bf16split"])
@pytest.mark.parametrize("rounds", [2, 4, 7])
def test_rounds_circuits_against_dense(dtype, rounds):
    n = 10
    rng = np.random.default_rng(300 + rounds)
    circ = inputs.rounds_circuit(n, rounds, rng)
    terms = inputs.random_pauli_terms(n, 40, 4, rng)
    m = tnmps.MPSBatch(n, 32, 1, dtype=dtype, max_params=0, eps=1e-12)
    m.apply_circuit(circ, None)
    e, pt = m.expect(tnmps.PauliSum(n, terms), per_term=True)
    m.check()
    ref = OE.term_values_dense(n, circ, np.zeros(0), terms)
    tol = 1e-10 if dtype == "c128" else 1e-4
    assert np.max(np.abs(pt[0] - ref)) <= tol
    om = OM.MPS(n, 32, 1e-12).run(circ, np.zeros(0))
    if dtype == "c128":
        assert list(m.bond_dims()[0]) == om.bond_dims()
    if rounds == 2:  # Sec. V.A: two rounds keep every bond at <= 4
        assert m.bond_dims().max() <= 4
