"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs."""
import numpy as np
import pytest

from oracle import energy as OE
from oracle import mps as OM
from oracle import statevector as SV
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

# tolerances: FP64 form against the oracle (absolute, per term); FP32 form
# against |dE| <= 1e-6 * sum|c_k| (the accuracy target of the mixed form)
TOL64 = 1e-10


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


def gpu_values(n, chi, eps, circ, thetas, terms, dtype="c128"):
    B = thetas.shape[0] if thetas is not None and np.ndim(thetas) == 2 else 1
    P = thetas.shape[-1] if thetas is not None else 0
    m = tnmps.MPSBatch(n, chi, B, dtype=dtype, max_params=P, eps=eps)
    m.apply_circuit(circ, thetas)
    ps = tnmps.PauliSum(n, terms)
    e, pt = m.expect(ps, per_term=True)
    return m, e, pt


@pytest.mark.parametrize("rep", [0, 1])
def test_hea8_c128_matches_dense(rep):
    wl = inputs.workload("hea8", rep)
    th = wl["thetas"]
    m, e, pt = gpu_values(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"])
    dims = m.bond_dims()
    for b in range(th.shape[0]):
        ref = OE.term_values_dense(wl["n"], wl["circuit"], th[b], wl["terms"])
        assert np.max(np.abs(pt[b] - ref)) <= TOL64
        assert abs(e[b] - OE.energy_from_values(wl["terms"], ref)) <= TOL64 * sum_abs(wl["terms"])
        om = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], th[b])
        assert list(dims[b]) == om.bond_dims()
    assert np.all(m.discarded() < 1e-20)


def test_hea8_c64_within_mixed_tolerance():
    wl = inputs.workload("hea8", 0)
    th = wl["thetas"]
    m, e, pt = gpu_values(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"], "c64")
    for b in range(th.shape[0]):
        ref = OE.energy(wl["n"], wl["circuit"], th[b], wl["terms"], "dense")
        assert abs(e[b] - ref) <= 1e-6 * sum_abs(wl["terms"])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_h2_ansatz_closed_form_grid(dtype):
    """The paper's two-qubit VQE ansatz on its 100-point grid in [-pi, pi],
    one grid point per batch member, against the dense oracle."""
    rng = np.random.default_rng(42)
    terms = inputs.all_two_qubit_terms(rng)
    circ, _ = inputs.h2_ansatz()
    grid = np.linspace(-np.pi, np.pi, 100).reshape(100, 1)
    m, e, _ = gpu_values(2, 4, 1e-12, circ, grid, terms, dtype)
    tol = TOL64 if dtype == "c128" else 1e-6
    for b in range(100):
        ref = OE.energy(2, circ, grid[b], terms, "dense")
        assert abs(e[b] - ref) <= tol * sum_abs(terms)


def test_non_adjacent_reversed_and_single_qubit_gates():
    rng = np.random.default_rng(5)
    n = 7
    circ = [("H", q, -1, -1, 0.0, 1.0) for q in range(0, n, 2)]
    circ += [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    circ += [("CNOT", 0, 5, -1, 0.0, 1.0), ("CZ", 6, 2, -1, 0.0, 1.0), ("S", 3, -1, -1, 0, 1),
             ("CNOT", 4, 3, -1, 0.0, 1.0), ("SWAP", 1, 6, -1, 0.0, 1.0),
             ("RX", 3, -1, n, 0.3, 2.0), ("CNOT", 6, 0, -1, 0.0, 1.0), ("T", 2, -1, -1, 0, 1),
             ("Y", 5, -1, -1, 0, 1), ("RZ", 1, -1, n + 1, 0.0, 1.0)]
    th = rng.uniform(-np.pi, np.pi, (3, n + 2))
    terms = inputs.random_pauli_terms(n, 40, 4, rng)
    m, e, pt = gpu_values(n, 16, 1e-12, circ, th, terms)
    for b in range(3):
        ref = OE.term_values_dense(n, circ, th[b], terms)
        assert np.max(np.abs(pt[b] - ref)) <= TOL64


def test_single_qubit_only_and_identity_term():
    n = 5
    th = np.array([[0.3, -1.1, 2.0, 0.7, -0.4]])
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    terms = [(0.5, (), ()), (1.0, (0,), (3,)), (1.0, (1, 3), (1, 3)), (2.0, (4,), (2,))]
    m, e, pt = gpu_values(n, 4, 1e-12, circ, th, terms)
    ref = [1.0, np.cos(0.3), np.sin(-1.1) * np.cos(0.7), 0.0]
    assert np.allclose(pt[0], ref, atol=1e-13)
    assert np.all(m.bond_dims() == 1)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ghz_n40(dtype):
    n = 40
    circ = [("H", 0, -1, -1, 0.0, 1.0)] + [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    terms = [(1.0, tuple(range(n)), (1,) * n), (1.0, tuple(range(n)), (2, 2) + (1,) * (n - 2)),
             (1.0, (3, 31), (3, 3)), (1.0, (17,), (3,))]
    m, e, pt = gpu_values(n, 8, 1e-10, circ, None, terms, dtype)
    tol = 1e-12 if dtype == "c128" else 1e-6
    assert np.allclose(pt[0], [1, -1, 1, 0], atol=tol)
    assert np.all(m.bond_dims() == 2)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_heis40_against_oracle_mps(dtype):
    wl = inputs.workload("heis40")
    B = 6
    th = wl["thetas"][:B]
    m, e, pt = gpu_values(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, wl["terms"], dtype)
    dims = m.bond_dims()
    scale = sum_abs(wl["terms"])
    for b in range(2):
        vals, om = OE.term_values_mps(wl["n"], wl["circuit"], th[b], wl["terms"], wl["chi_max"],
                                      wl["eps"])
        eref = OE.energy_from_values(wl["terms"], vals)
        if dtype == "c128":
            assert np.max(np.abs(pt[b] - vals)) <= TOL64
            assert list(dims[b]) == om.bond_dims()
        else:
            assert abs(e[b] - eref) <= 1e-6 * scale


@pytest.mark.parametrize("dtype,shape", [("c128", (7, 5)), ("c128", (33, 17)), ("c128", (64, 64)),
                                         ("c128", (200, 130)), ("c128", (256, 256)),
                                         ("c128", (96, 160)), ("c64", (256, 256)),
                                         ("c64", (130, 70)), ("c64", (512, 300))])
def test_jacobi_svd_against_lapack(dtype, shape):
    m, n = shape
    rng = np.random.default_rng(m * 1000 + n)
    B = 3
    A = rng.normal(size=(B, m, n)) + 1j * rng.normal(size=(B, m, n))
    A[1] = A[1] * np.logspace(0, -9, n)[None, :]          # graded columns
    A[2, :, n // 2:] = A[2, :, : n - n // 2] @ rng.normal(size=(n - n // 2, n - n // 2)) * 0  # rank-deficient
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    lda = m + 3
    buf = np.zeros((B, n, lda), dtype=np.complex128)
    buf[:, :, :m] = np.transpose(A, (0, 2, 1))
    a = torch.tensor(buf, dtype=tdt, device="cuda")
    sig = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    sw = torch.zeros(B, dtype=torch.int32, device="cuda")
    tnmps.jacobi_svd_dev(a, m, n, sig, sw)
    torch.cuda.synchronize()
    W = np.transpose(a.cpu().numpy()[:, :, :m], (0, 2, 1)).astype(np.complex128)
    s = sig.cpu().numpy()
    # FP64: LAPACK-level agreement. FP32: every column takes ~N rotations per
    # sweep, each rounding at 2^-24, so singular values drift by up to ~1e-4
    # of sigma_max and orthogonality stops at ~(sqrt(m)+16) 2^-24 (column-relative).
    tol, orth_tol, floor = (1e-12, 1e-13, 1e-10) if dtype == "c128" else (1e-4, 2e-5, 1e-3)
    for b in range(B):
        ref = np.linalg.svd(A[b], compute_uv=False)
        got = np.sort(s[b])[::-1][: len(ref)]
        assert np.max(np.abs(got - ref)) <= tol * ref[0]
        # W = A V: same Gram from the left
        assert np.linalg.norm(W[b] @ W[b].conj().T - A[b] @ A[b].conj().T) <= tol * 10 * ref[0] ** 2
        # columns mutually orthogonal (relative to their norms)
        nrm = np.linalg.norm(W[b], axis=0)
        keep = nrm > floor * ref[0]
        Wk = W[b][:, keep] / nrm[keep]
        G = Wk.conj().T @ Wk
        assert np.max(np.abs(G - np.eye(G.shape[0]))) <= orth_tol
    assert np.all(sw.cpu().numpy() > 0)


def test_injected_fault_and_bad_arguments():
    m = tnmps.MPSBatch(4, 4, 1)
    m.inject(1, 7)
    with pytest.raises(tnmps.TnmpsError) as ei:
        m.apply_circuit([("H", 0, -1, -1, 0, 1)])
    assert ei.value.status == 7
    m.reset()
    with pytest.raises(tnmps.TnmpsError):
        m.apply_circuit([("CNOT", 0, 0, -1, 0, 1)])
    with pytest.raises(tnmps.TnmpsError):
        m.apply_circuit([("RY", 9, -1, -1, 0, 1)])
    with pytest.raises(tnmps.TnmpsError):
        m.apply_circuit([("RY", 0, -1, 3, 0, 1)], np.zeros(2))  # param index beyond n_params
