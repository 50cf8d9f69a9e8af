"""GPU parity of super-gate application by overlap maximisation: the CUDA
path (through the C ABI) against the oracle on the same seeded states, the
exact state-vector result and a closed form."""
import copy

import numpy as np
import pytest

from oracle import gates as G
from oracle import mps as OM
from oracle import statevector as SV
from oracle import supergate as OSG
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

BLOCK = [("CNOT", 2, 5, -1, 0.0, 1.0), ("RY", 3, -1, 0, 0.0, 1.0), ("CZ", 6, 3, -1, 0.0, 1.0),
         ("SWAP", 4, 2, -1, 0.0, 1.0), ("H", 5, -1, -1, 0.0, 1.0), ("RZ", 1, -1, 1, 0.0, 1.0),
         ("CNOT", 6, 1, -1, 0.0, 1.0), ("RX", 4, -1, -1, 0.7, 1.0), ("CNOT", 1, 2, -1, 0.0, 1.0)]
BLOCK_THETA = np.array([0.9, -1.3])
DTYPES = ["c128", "c64", "c64_bf16split"]
# fidelity and state agreement: FP64 form / FP32 contraction forms
FTOL = {"c128": 1e-10, "c64": 2e-5, "c64_bf16split": 2e-5}


def gpu_sites(m, b):
    return [m.site(b, i) for i in range(m.n)]


def overlap(A, B):
    """<A|B> of two MPS given as lists of (D, 2, D) tensors."""
    L = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        L = np.einsum("xy,xsa,ysb->ab", L, a.conj(), b)
    return complex(L[0, 0])


def dense(sites):
    v = sites[0].reshape(2, -1)
    for A in sites[1:]:
        v = np.einsum("xm,msb->xsb", v, A).reshape(-1, A.shape[2])
    n = len(sites)
    return np.transpose(v.reshape((2,) * n), tuple(range(n - 1, -1, -1))).reshape(-1)


def states(n, layers, chi, B, seed, dtype, eps):
    rng = np.random.default_rng(seed)
    circ, P = inputs.hea_circuit(n, layers, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, (B, P))
    m = tnmps.MPSBatch(n, chi, B, dtype=dtype, max_params=P, eps=eps)
    m.apply_circuit(circ, th)
    oms = [OM.MPS(n, chi, eps).run(circ, th[b]) for b in range(B)]
    return m, oms, circ, th


@pytest.mark.parametrize("dtype", DTYPES)
def test_block_matches_oracle(dtype):
    n, B = 8, 2
    m, oms, _, _ = states(n, 3, 16, B, 21, dtype, 1e-6)
    w0 = m.discarded()
    sg = tnmps.Supergate(n, BLOCK, BLOCK_THETA)
    F, F0, info = m.apply_supergate(sg, chi_max=4, target=1e-10, tol=-1.0, max_sweeps=3)
    assert info == {"sweeps": 3, "stages": 1, "chi": 4}
    dims = m.bond_dims()
    w1 = m.discarded()
    for b in range(B):
        phi, f, hist, chi, f0 = OSG.apply_supergate(oms[b], BLOCK, BLOCK_THETA, chi_max=4,
                                                    target=1e-10, tol=-1.0, max_sweeps=3)
        assert len(hist) == 3 and chi == 4
        assert abs(F[b] - f) <= FTOL[dtype]
        assert abs(F0[b] - f0) <= FTOL[dtype]
        assert F[b] > F0[b] + 1e-4  # the sweeps improve on gate-by-gate truncation
        assert list(dims[b]) == phi.bond_dims()
        ov = abs(overlap(gpu_sites(m, b), phi.tensors))
        assert ov >= 1.0 - FTOL[dtype]
        assert abs((w1[b] - w0[b]) - (1.0 - F[b])) <= 1e-9


@pytest.mark.parametrize("dtype", DTYPES)
def test_exact_without_truncation(dtype):
    n = 8
    m, oms, circ, th = states(n, 2, 64, 1, 23, dtype, 1e-10)
    sg = tnmps.Supergate(n, BLOCK, BLOCK_THETA)
    target = 1e-12 if dtype == "c128" else 1e-5
    F, _, info = m.apply_supergate(sg, chi_max=64, target=target, tol=1e-12)
    assert info["stages"] > 1  # step (6) had to grow the bonds of the copy
    assert abs(F[0] - 1.0) <= FTOL[dtype]
    psi = SV.run_circuit(n, circ, th[0])
    for gate in BLOCK:
        if G.is_two_qubit(gate):
            psi = SV.apply_2q(psi, n, G.two_qubit(gate[0]), gate[1], gate[2])
        else:
            psi = SV.apply_1q(psi, n, G.one_qubit_matrix(gate, BLOCK_THETA), gate[1])
    v = dense(gpu_sites(m, 0))
    assert abs(abs(np.vdot(v, psi)) - 1.0) <= 10 * FTOL[dtype]
    np.testing.assert_allclose(v, psi, atol=1e-9 if dtype == "c128" else 2e-3)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_distant_cnot_closed_form(dtype):
    n = 6
    cnot = tnmps.Supergate(n, [("CNOT", 0, 4, -1, 0.0, 1.0)])
    m = tnmps.MPSBatch(n, 8, 1, dtype=dtype, eps=1e-10)
    m.apply_circuit([("H", 0, -1, -1, 0.0, 1.0)])
    F, _, info = m.apply_supergate(cnot, chi_max=1)
    assert abs(F[0] - 0.5) <= FTOL[dtype] and info["chi"] == 1
    m.reset()
    m.apply_circuit([("H", 0, -1, -1, 0.0, 1.0)])
    F, _, info = m.apply_supergate(cnot, chi_max=4, target=1e-6)
    assert abs(F[0] - 1.0) <= FTOL[dtype]
    assert info["chi"] == 2 and info["stages"] == 2
    assert list(m.bond_dims()[0]) == [2, 2, 2, 2, 1]
    v = dense(gpu_sites(m, 0))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[(1 << 0) | (1 << 4)] = 1 / np.sqrt(2)
    assert abs(abs(np.vdot(v, ref)) - 1.0) <= 1e-6


def test_single_adjacent_gate_is_eckart_young():
    n = 6
    m, oms, _, _ = states(n, 3, 8, 1, 25, "c128", 1e-12)
    gates = [("RY", 2, -1, 0, 0.0, 1.0), ("CNOT", 2, 3, -1, 0.0, 1.0), ("RX", 3, -1, 1, 0.0, 1.0)]
    th = np.array([0.4, 1.1])
    F, F0, _ = m.apply_supergate(tnmps.Supergate(n, gates, th), chi_max=2)
    ref = copy.deepcopy(oms[0])
    ref.chi_max = 2
    ref.run(gates, th)
    w = ref.step_weights[-1]
    assert w > 1e-3
    assert abs(F[0] - (1.0 - w)) <= 1e-10 and abs(F0[0] - (1.0 - w)) <= 1e-10


def test_n40_window_matches_oracle():
    n, B = 40, 2
    m, oms, _, _ = states(n, 4, 16, B, 27, "c64", 1e-6)
    block = [("CNOT", 17, 21, -1, 0.0, 1.0), ("RY", 19, -1, 0, 0.0, 1.0),
             ("CZ", 22, 18, -1, 0.0, 1.0), ("H", 20, -1, -1, 0.0, 1.0),
             ("CNOT", 18, 19, -1, 0.0, 1.0), ("SWAP", 20, 17, -1, 0.0, 1.0)]
    th = np.array([0.8])
    sg = tnmps.Supergate(n, block, th)
    assert (sg.first, sg.last) == (17, 22)
    F, F0, info = m.apply_supergate(sg, chi_max=8, target=1e-10, tol=-1.0, max_sweeps=2)
    terms = [(1.0, [19], [3]), (0.5, [20, 21], [1, 1]), (-0.7, [17, 22], [2, 3]),
             (0.3, [5, 30], [3, 3])]
    _, pt = m.expect(tnmps.PauliSum(n, terms), per_term=True)
    for b in range(B):
        phi, f, _, _, f0 = OSG.apply_supergate(oms[b], block, th, chi_max=8, target=1e-10,
                                               tol=-1.0, max_sweeps=2)
        assert abs(F[b] - f) <= FTOL["c64"] and abs(F0[b] - f0) <= FTOL["c64"]
        for k, (_, sites, paulis) in enumerate(terms):
            ref = phi.expect_pauli(sites, paulis).real
            assert abs(pt[b, k] - ref) <= 1e-5


def test_bad_arguments():
    m = tnmps.MPSBatch(8, 8, 1, dtype="c64")
    with pytest.raises(tnmps.TnmpsError):
        m.apply_supergate(tnmps.Supergate(8, BLOCK, BLOCK_THETA), chi_max=0)
    with pytest.raises(tnmps.TnmpsError):
        m.apply_supergate(tnmps.Supergate(10, BLOCK, BLOCK_THETA), chi_max=4)
    with pytest.raises(tnmps.TnmpsError):
        m.apply_supergate(tnmps.Supergate(8, BLOCK, BLOCK_THETA), chi_max=9)


def test_chi128_window_matches_oracle():
    # full size: the chi = 128 benchmark states (40 qubits, 10 layers) and the
    # measured six-qubit block; the oracle fits the first two states
    wl = inputs.workload("chi128")
    B = 2
    th = wl["thetas"][:B]
    m = tnmps.MPSBatch(40, 128, B, dtype="c64_bf16split", max_params=wl["n_params"],
                       eps=wl["eps"])
    m.apply_circuit(wl["circuit"], th)
    block, bth = inputs.supergate_block(17, inputs.rng_for(5, 11))
    kw = dict(chi_max=128, target=1e-10, tol=-1.0, max_sweeps=2)
    F, F0, info = m.apply_supergate(tnmps.Supergate(40, block, bth), **kw)
    assert info == {"sweeps": 2, "stages": 1, "chi": 128}
    terms = [(1.0, [19], [3]), (0.5, [18, 21], [1, 1]), (-0.7, [17, 22], [2, 3])]
    _, pt = m.expect(tnmps.PauliSum(40, terms), per_term=True)
    for b in range(B):
        om = OM.MPS(40, 128, wl["eps"]).run(wl["circuit"], th[b])
        phi, f, _, _, f0 = OSG.apply_supergate(om, block, bth, **kw)
        assert abs(F0[b] - f0) <= 1e-5 and abs(F[b] - f) <= 1e-5
        assert F[b] > F0[b] + 0.05
        for k, (_, sites, paulis) in enumerate(terms):
            assert abs(pt[b, k] - phi.expect_pauli(sites, paulis).real) <= 1e-4


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_window_at_the_last_site_then_circuit(dtype):
    # window reaching site n-1, a second super-gate, then an ordinary circuit and
    # the energy: the context's gauge and bond bookkeeping after a fit must hold
    n, B = 9, 2
    m, oms, _, _ = states(n, 3, 16, B, 29, dtype, 1e-10)
    sg1 = [("CNOT", 8, 5, -1, 0.0, 1.0), ("RY", 6, -1, 0, 0.0, 1.0), ("SWAP", 7, 5, -1, 0.0, 1.0)]
    sg2 = [("CZ", 1, 4, -1, 0.0, 1.0), ("H", 2, -1, -1, 0.0, 1.0), ("CNOT", 3, 2, -1, 0.0, 1.0)]
    th = np.array([1.1])
    kw = dict(target=1e-10, tol=-1.0, max_sweeps=2)
    F1, _, i1 = m.apply_supergate(tnmps.Supergate(n, sg1, th), chi_max=6, **kw)
    F2, _, i2 = m.apply_supergate(tnmps.Supergate(n, sg2, None), chi_max=5, **kw)
    tail = [("RX", q, -1, -1, 0.3 * (q + 1), 1.0) for q in range(n)] + \
           [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    m.apply_circuit(tail)
    terms = [(1.0, [0], [3]), (0.4, [4, 5], [1, 2]), (-0.6, [7, 8], [3, 3]), (0.2, [2, 6], [2, 1])]
    e, pt = m.expect(tnmps.PauliSum(n, terms), per_term=True)
    tol = FTOL[dtype]
    for b in range(B):
        p1, f1, _, _, _ = OSG.apply_supergate(oms[b], sg1, th, chi_max=6, **kw)
        p2, f2, _, _, _ = OSG.apply_supergate(p1, sg2, None, chi_max=5, **kw)
        assert abs(F1[b] - f1) <= tol and abs(F2[b] - f2) <= tol
        p2.chi_max = 16
        p2.run(tail, None)
        ref = np.array([p2.expect_pauli(s, p).real for _, s, p in terms])
        assert np.max(np.abs(pt[b] - ref)) <= (1e-9 if dtype == "c128" else 2e-5)
    assert i1["chi"] == 6 and i2["chi"] == 5


def test_one_qubit_window_applies_exactly():
    n = 6
    m, oms, circ, th = states(n, 2, 8, 2, 31, "c128", 1e-12)
    gates = [("RY", 3, -1, 0, 0.0, 1.0), ("H", 3, -1, -1, 0.0, 1.0)]
    F, F0, info = m.apply_supergate(tnmps.Supergate(n, gates, np.array([0.4])), chi_max=8)
    assert np.all(F == 1.0) and info["sweeps"] == 0
    for b in range(2):
        psi = SV.run_circuit(n, circ, th[b])
        psi = SV.apply_1q(psi, n, G.ry(0.4), 3)
        psi = SV.apply_1q(psi, n, G.H, 3)
        v = dense(gpu_sites(m, b))
        assert abs(abs(np.vdot(v, psi)) - 1.0) <= 1e-10
