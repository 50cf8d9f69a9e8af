"""Truncation semantics on the GPU circuit path against the FP64 oracle: the
cutoff rule of Sec. IV (singular values below eps ||sigma|| dropped, the
paper's default eps = 1e-4), the chi_max cap, and the discarded weight
w = sum of dropped sigma^2 / sum sigma^2 per step, accumulated per state.

The oracle's discarded weight is pinned to the truncation error of each step
(``tests/test_oracle_mps.py``: ||psi - psi_trunc||^2 = w), so matching it pins
the library's accounting to the same definition. Every case checks the
oracle's decision margins first (``oracle.mps.cut_margin``) so that the
expected truncation is unique at each precision."""
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

DTYPES = ["c128", "c64", "c64_bf16split"]
# per dtype: per-term, relative discarded weight, smallest decision margin the
# arithmetic resolves (relative to sigma_0), and an absolute floor on the
# discarded weight per truncating step: a dropped value sigma carries an
# absolute error d ~ sqrt(M) u sigma_0 from the FP32 Jacobi (u = 2^-24, M <= 16
# rows here: d <= 2.4e-7), so sigma^2 is off by up to 2 sigma d + d^2 -- about
# 1e-11 for the sigma ~ 3e-5 that eps = 1e-4 drops
BARS = {"c128": (1e-10, 1e-10, 1e-12, 0.0), "c64": (1e-4, 1e-4, 1e-5, 1e-11),
        "c64_bf16split": (1e-4, 1e-4, 1e-5, 1e-11)}


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


def gpu_run(n, chi, eps, circ, th, terms, dtype):
    m = tnmps.MPSBatch(n, chi, th.shape[0], dtype=dtype, max_params=th.shape[1], eps=eps)
    m.apply_circuit(circ, th)
    e, pt = m.expect(tnmps.PauliSum(n, terms), per_term=True)
    m.check()
    return m.bond_dims(), m.discarded(), e, pt


def compare(n, chi, eps, circ, th, terms, dtype, expect_cut=True):
    tol_p, tol_w, margin, w_floor = BARS[dtype]
    dims, w, e, pt = gpu_run(n, chi, eps, circ, th, terms, dtype)
    for b in range(th.shape[0]):
        vals, om = OE.term_values_mps(n, circ, th[b], terms, chi, eps)
        cm = np.array(om.cut_margins)
        assert cm[:, 0].min() > margin and cm[:, 1].min() > margin, (b, cm.min(axis=0))
        if expect_cut:
            assert om.discarded > 0, "the case must truncate something"
        msg = (f"{dtype} b={b} dims {list(dims[b])} vs {om.bond_dims()}, w {w[b]:.6e} vs "
               f"{om.discarded:.6e}, max|dP| {np.abs(pt[b] - vals).max():.2e}")
        assert list(dims[b]) == om.bond_dims(), msg
        cuts = int(np.count_nonzero(np.array(om.step_weights) > 0))
        assert abs(w[b] - om.discarded) <= tol_w * om.discarded + w_floor * cuts + 1e-30, msg
        assert np.abs(pt[b] - vals).max() <= tol_p, msg
        tol_e = 1e-10 if dtype == "c128" else 1e-6
        assert abs(e[b] - OE.energy_from_values(terms, vals)) <= tol_e * sum_abs(terms), msg


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("chi", [3, 4, 6])
def test_binding_chi_cap_discarded_weight(dtype, chi):
    """10 qubits, 4 Ry/Rz + ladder layers, bonds capped at chi (the cap cuts
    up to 80 % of the weight): bond dimensions, cumulative discarded weight
    and term values against the oracle."""
    n = 10
    circ, P = inputs.hea_circuit(n, 4, ("RY", "RZ"))
    th = inputs.thetas(3, P, np.random.default_rng(78))
    terms = inputs.heisenberg_terms(n, np.random.default_rng(79)) + \
        inputs.random_pauli_terms(n, 40, 4, np.random.default_rng(80))
    compare(n, chi, 1e-12, circ, th, terms, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_paper_default_cutoff_on_weakly_entangled_hea(dtype):
    """The paper's default cutoff eps = 1e-4 on a 10-qubit HEA whose Ry angles
    are small (Schmidt values between 1e-5 and 1e-3 appear): the cut removes
    values (bond 7 instead of 8) without any cap."""
    n = 10
    circ, P = inputs.hea_circuit(n, 3, ("RY", "RZ"))
    th = inputs.thetas(3, P, np.random.default_rng(79)) * 0.003
    th[:, 1::2] = inputs.thetas(3, P, np.random.default_rng(80))[:, 1::2]
    terms = inputs.random_pauli_terms(n, 60, 4, np.random.default_rng(81))
    compare(n, 64, 1e-4, circ, th, terms, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("s,expected_dim", [(5e-5, 1), (2e-4, 2)])
def test_paper_default_cutoff_two_qubit_schmidt_pair(dtype, s, expected_dim):
    """cos(a)|00> + sin(a)|11> has Schmidt values (cos a, sin a): eps = 1e-4
    drops sin a = 5e-5 (weight sin^2 a, <Z0> = 1 after renormalisation) and
    keeps 2e-4."""
    a = np.arcsin(s)
    circ = [("RY", 0, -1, 0, 0.0, 1.0), ("CNOT", 0, 1, -1, 0.0, 1.0)]
    th = np.array([[2 * a]])
    dims, w, e, pt = gpu_run(2, 8, 1e-4, circ, th, [(1.0, (0,), (3,)), (1.0, (0, 1), (1, 1))],
                             dtype)
    assert dims[0, 0] == expected_dim
    if expected_dim == 1:
        assert abs(w[0] - s * s) <= (1e-12 if dtype == "c128" else 1e-3) * s * s
        tol = 1e-12 if dtype == "c128" else 1e-6
        assert abs(pt[0, 0] - 1.0) <= tol and abs(pt[0, 1]) <= tol
    else:
        assert w[0] <= 1e-20
        assert abs(pt[0, 0] - np.cos(2 * a)) <= (1e-12 if dtype == "c128" else 1e-6)
        assert abs(pt[0, 1] - np.sin(2 * a)) <= (1e-12 if dtype == "c128" else 1e-6)
