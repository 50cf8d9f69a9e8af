"""Every launch shape the autotuner can choose computes the same state and
energies: the chi = 128 benchmark workload (its bonds grow through 2..128, so
all three complex64 Jacobi block-size classes run) in each candidate
configuration against the FP64 oracle on the same theta row; then the tuner
itself on a small workload."""
import numpy as np
import pytest

from oracle import energy as OE
from oracle import mps as OM
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import autotune, tnmps  # noqa: E402

CANDIDATES = [
    {"jacobi_shape": [0, 0, 0], "gemm_stages": 0, "sweep_fused": 0},
    {"jacobi_shape": [1, 0, 0], "gemm_stages": 0, "sweep_fused": 0},
    {"jacobi_shape": [0, 1, 0], "gemm_stages": 0, "sweep_fused": 0},
    {"jacobi_shape": [0, 0, 1], "gemm_stages": 0, "sweep_fused": 0},
    {"jacobi_shape": [1, 1, 1], "gemm_stages": 2, "sweep_fused": 1},
    {"jacobi_shape": [0, 0, 0], "gemm_stages": 3, "sweep_fused": 1},
]


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


@pytest.fixture(scope="module")
def reference():
    wl = inputs.workload("chi128")
    rand = wl["terms_random"][:40]
    m = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], wl["thetas"][0])
    assert np.array(m.cut_margins)[:, 1].min() > 1e-5
    heis = np.array([m.expect_pauli(s, p).real for _, s, p in wl["terms"]])
    rv = np.array([m.expect_pauli(s, p).real for _, s, p in rand])
    return wl, rand, heis, rv


@pytest.mark.parametrize("dtype", ["c64", "c64_bf16split"])
@pytest.mark.parametrize("cand", range(len(CANDIDATES)))
def test_every_candidate_matches_oracle(reference, dtype, cand):
    wl, rand, heis, rv = reference
    cfg = CANDIDATES[cand]
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], 1, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.set_tuning(**cfg)
    assert m.get_tuning() == cfg
    m.apply_circuit(wl["circuit"], wl["thetas"][:1])
    eh, pth = m.expect(tnmps.PauliSum(wl["n"], wl["terms"]), per_term=True)
    er, ptr = m.expect(tnmps.PauliSum(wl["n"], rand), per_term=True)
    m.check()
    assert np.abs(pth[0] - heis).max() <= 1e-4 and np.abs(ptr[0] - rv).max() <= 1e-4
    assert abs(eh[0] - OE.energy_from_values(wl["terms"], heis)) <= 1e-6 * sum_abs(wl["terms"])
    assert abs(er[0] - OE.energy_from_values(rand, rv)) <= 1e-6 * sum_abs(rand)


def test_bad_tuning_rejected():
    m = tnmps.MPSBatch(4, 4, 1, dtype="c64")
    for bad in ({"jacobi_shape": [2, 0, 0]}, {"gemm_stages": 1}, {"gemm_stages": 4},
                {"sweep_fused": 2}):
        with pytest.raises(tnmps.TnmpsError) as ei:
            m.set_tuning(**bad)
        assert ei.value.status == 1
    assert m.get_tuning() == {"jacobi_shape": [0, 0, 0], "gemm_stages": 0, "sweep_fused": 0}
    for bad in (0.5, 5000.0, float("nan")):
        with pytest.raises(tnmps.TnmpsError) as ei:
            m.set_svd_tolerance(bad)
        assert ei.value.status == 1
    for bad in (-1, 2):
        with pytest.raises(tnmps.TnmpsError) as ei:
            m.set_svd_precondition(bad)
        assert ei.value.status == 1


@pytest.mark.parametrize("chunk", [0, 3])
def test_fused_sweep_bit_identical_to_two_launches(chunk):
    """Both steps of each trie level in one launch (T in per-CTA slots) give
    exactly the two-launch values: the same MMAs and epilogues, only the
    launch structure and the T buffers differ. 5 states of 9-layer 40-qubit
    states (middle bonds at 128), 400 random strings, ragged state chunks."""
    wl = inputs.workload("chi128")
    circ, P = inputs.hea_circuit(40, 9, ("RY", "RZ"))
    th = inputs.thetas(5, P, np.random.default_rng(9))
    m = tnmps.MPSBatch(40, 128, 5, dtype="c64_bf16split", max_params=P, eps=1e-10)
    m.apply_circuit(circ, th)
    ps = tnmps.PauliSum(40, wl["terms_random"][:400])
    out = []
    for fused in (0, 1):
        m.set_tuning(sweep_fused=fused)
        out.append(m.expect(ps, per_term=True, chunk=chunk))
        m.check()
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])


def test_tuner_picks_a_candidate_and_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("TNMPS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    wl = inputs.workload("heis40")
    B = 8
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], B, dtype="c64_bf16split",
                       max_params=wl["n_params"], eps=wl["eps"])
    gates_c = tnmps.gate_array(wl["circuit"])
    th = torch.tensor(wl["thetas"][:B], dtype=torch.float64, device="cuda")
    ps = tnmps.PauliSum(wl["n"], wl["terms"])
    rep = autotune.tune_context(m, gates_c, th, {"heis": ps}, chunk_candidates=(2, 4))
    assert not rep["cached"] and m.get_tuning() == rep["tuning"]
    # a candidate replaces the choice only when more than 1 % faster
    assert min(t["circuit_s"] for t in rep["trials"] if "circuit_s" in t) >= \
        0.99 * rep["circuit_s"]["tuned"] - 1e-12
    assert rep["chunk"]["heis"] in (0, 2, 4)
    again = autotune.tune_context(m, gates_c, th, {"heis": ps})
    assert again["cached"] and again["tuning"] == rep["tuning"]
    m.reset()
    m.apply_circuit_dev(gates_c, th)
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    m.expect_dev(ps, e, chunk=rep["chunk"]["heis"])
    torch.cuda.synchronize()
    for b in range(2):
        ref = OE.energy(wl["n"], wl["circuit"], wl["thetas"][b], wl["terms"], "mps",
                        wl["chi_max"], wl["eps"])
        assert abs(e[b].item() - ref) <= 1e-6 * sum_abs(wl["terms"])
