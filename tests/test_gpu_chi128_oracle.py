"""The chi = 128 throughput workload against the FP64 oracle MPS.

The workload the benchmark times: 40 qubits, 10 layers of (Ry, Rz on every
qubit; CNOT ladder), chi_max 128 with the cap binding in every middle bond
(layers 8-10 truncate a full 256 x 256 two-site block at every interior gate),
cutoff 1e-10. Two of its theta rows are simulated in every arithmetic form and
compared with ``oracle/mps.py`` (LAPACK SVD, rule R, per-term full sweeps) on
the same rows, for both term sets of the metric: the 157-term Heisenberg
chain and a subset of the 2000 random strings of weight <= 4 (in the
BF16-split form both go through the tensor-core sweeps).

Bars:
* complex128: the oracle's bond dimensions, its cumulative discarded weight
  (1e-10 relative) and every term value (1e-10 absolute), provided no step of
  the oracle run sits within 1e-8 sigma_0 of a tie at the chi_max cut or
  within 1e-12 sigma_0 of the cutoff (Sec. IV cutoff rule; a tie leaves the
  truncated state non-unique, and the test then checks the energy only);
* complex64 and BF16-split: |dE| <= 1e-6 sum_k |c_k| for both term sets (the
  accuracy target of the mixed forms), every term within 1e-4, the discarded
  weight within 1e-4 relative (FP32 singular values carry ~1e-6 relative
  error per step), provided the chi_max cut has a gap of at least 1e-5 sigma_0
  at every step (the FP32 SVD's resolution); also with the Jacobi tolerance
  factor 64 that the benchmark uses.

Every case runs with the Jacobi on L of Theta = L Q^H (the default) and the
complex128 and complex64 forms also with the Jacobi on Theta itself; both
must meet the same bars, and the LQ form needs fewer sweeps.
"""
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

ROWS = 2
N_RANDOM = 50


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


@pytest.fixture(scope="module")
def reference():
    wl = inputs.workload("chi128")
    rand = wl["terms_random"][:N_RANDOM]
    rows = []
    for b in range(ROWS):
        m = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], wl["thetas"][b])
        cm = np.array(m.cut_margins)
        rows.append({
            "dims": m.bond_dims(), "w": m.discarded,
            "d_cut": float(cm[:, 0].min()), "d_cap": float(cm[:, 1].min()),
            "heis": np.array([m.expect_pauli(s, p).real for _, s, p in wl["terms"]]),
            "rand": np.array([m.expect_pauli(s, p).real for _, s, p in rand]),
        })
    return wl, rand, rows


SWEEPS = {}


@pytest.mark.parametrize("dtype,svd_tol,lq", [("c128", 1, 1), ("c64", 1, 1),
                                              ("c64_bf16split", 1, 1), ("c64_bf16split", 64, 1),
                                              ("c128", 1, 0), ("c64", 1, 0)])
def test_chi128_workload_against_oracle(reference, dtype, svd_tol, lq):
    """svd_tol 64: the Jacobi tolerance factor the benchmark runs with; lq:
    the Jacobi on L of Theta = L Q^H (1) or on Theta (0)."""
    wl, rand, rows = reference
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], ROWS, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.set_svd_tolerance(svd_tol)
    m.set_svd_precondition(lq)
    m.apply_circuit(wl["circuit"], wl["thetas"][:ROWS])
    st = m.stats()
    SWEEPS[(dtype, svd_tol, lq)] = st["jacobi_sweeps"] / st["svds"]
    eh, pth = m.expect(tnmps.PauliSum(wl["n"], wl["terms"]), per_term=True)
    er, ptr = m.expect(tnmps.PauliSum(wl["n"], rand), per_term=True)
    m.check()
    dims = m.bond_dims()
    w = m.discarded()
    sh, sr = sum_abs(wl["terms"]), sum_abs(rand)
    for b, r in enumerate(rows):
        assert dims[b].max() == wl["chi_max"]
        eh_ref = OE.energy_from_values(wl["terms"], r["heis"])
        er_ref = OE.energy_from_values(rand, r["rand"])
        dh, dr = np.abs(pth[b] - r["heis"]).max(), np.abs(ptr[b] - r["rand"]).max()
        msg = (f"{dtype} row {b}: max|dP| heis {dh:.3e} rand {dr:.3e}, |dE|/sum|c| heis "
               f"{abs(eh[b] - eh_ref) / sh:.3e} rand {abs(er[b] - er_ref) / sr:.3e}, "
               f"w {w[b]:.12f} vs {r['w']:.12f}, margins cut {r['d_cut']:.2e} cap {r['d_cap']:.2e}")
        if dtype == "c128":
            assert list(dims[b]) == r["dims"], msg
            if r["d_cap"] > 1e-8 and r["d_cut"] > 1e-12:
                assert dh <= 1e-10 and dr <= 1e-10, msg
                assert abs(w[b] - r["w"]) <= 1e-10 * r["w"], msg
                continue
        else:
            assert r["d_cap"] > 1e-5, msg
            assert dh <= 1e-4 and dr <= 1e-4, msg
            assert abs(w[b] - r["w"]) <= 1e-4 * r["w"], msg
        assert abs(eh[b] - eh_ref) <= 1e-6 * sh, msg
        assert abs(er[b] - er_ref) <= 1e-6 * sr, msg


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_lq_form_needs_fewer_sweeps(dtype):
    """Theta = L Q^H: the columns of L start closer to orthogonal (their Gram
    matrix is one QR-iteration step past Theta Theta^H), so the Jacobi on L
    converges in fewer sweeps than on Theta (both pass the oracle bars above)."""
    on, off = SWEEPS.get((dtype, 1, 1)), SWEEPS.get((dtype, 1, 0))
    if on is None or off is None:
        pytest.skip("runs after the parity cases of this module")
    assert on < off, (dtype, on, off)
