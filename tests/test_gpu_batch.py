"""Many heterogeneous circuits in one persistent launch, against the FP64
oracle and against the single-context path."""
import numpy as np
import pytest

from oracle import energy as OE
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402


def sum_abs(terms):
    return sum(abs(t[0]) for t in terms)


@pytest.mark.parametrize("block_cols", [32, 16])
def test_small_jobs_match_dense_oracle(block_cols):
    rng = np.random.default_rng(21)
    jobs = inputs.batch_jobs(24, rng, n_range=(2, 10), depth_range=(1, 4), chi_range=(16, 40),
                             terms_range=(1, 40))
    jobs[0]["terms"] = [(0.25, (), ())] + jobs[0]["terms"]   # identity term
    b = tnmps.Batch(jobs, cutoff=1e-12, ctas=7, block_cols=block_cols)
    e = b.run()
    for j, jb in enumerate(jobs):
        ref = OE.energy(jb["n"], jb["circuit"], jb["theta"], jb["terms"], "dense")
        assert abs(e[j] - ref) <= 1e-6 * max(1.0, sum_abs(jb["terms"])), j


def test_graph_replay_and_context_path_agree():
    rng = np.random.default_rng(5)
    jobs = inputs.batch_jobs(6, rng, n_range=(30, 40), depth_range=(3, 5), chi_range=(32, 64),
                             terms_range=(50, 200))
    b = tnmps.Batch(jobs, cutoff=1e-10)
    e1 = b.run()
    b.capture_graph()
    e2 = b.run()
    assert np.array_equal(e1, e2)                       # deterministic replay
    for j, jb in enumerate(jobs[:3]):
        m = tnmps.MPSBatch(jb["n"], jb["chi"], 1, dtype="c64", max_params=jb["n_params"],
                           eps=1e-10)
        m.apply_circuit(jb["circuit"], jb["theta"])
        ref = m.expect(tnmps.PauliSum(jb["n"], jb["terms"]))[0]
        assert abs(e1[j] - ref) <= 1e-6 * sum_abs(jb["terms"]), j


def test_configs2_sized_jobs_against_oracle():
    """Jobs of the heterogeneous-batch workload's sizes (16..64 qubits, depth
    2..8, chi_max 32..128 -- the cap binds in most of them) in one persistent
    launch, against the FP64 oracle MPS: energies within the mixed forms'
    target 1e-6 sum|c_k| and the discarded weights, for every job whose
    truncation is unique at FP32 resolution (no tie within 1e-5 sigma_0 at any
    chi_max cut)."""
    from oracle import mps as OM
    rng = np.random.default_rng(2024)
    jobs = inputs.batch_jobs(8, rng, terms_range=(50, 80))
    b = tnmps.Batch(jobs, cutoff=1e-10)
    b.launch()
    e, w = b.results()
    compared = truncated = 0
    for j, jb in enumerate(jobs):
        vals, om = OE.term_values_mps(jb["n"], jb["circuit"], jb["theta"], jb["terms"], jb["chi"],
                                      1e-10)
        cm = np.array(om.cut_margins)
        if cm[:, 1].min() <= 1e-5:
            continue                     # a near tie at the cap: the truncation is not unique
        compared += 1
        truncated += om.discarded > 0
        scale = sum_abs(jb["terms"])
        eref = OE.energy_from_values(jb["terms"], vals)
        assert abs(e[j] - eref) <= 1e-6 * scale, (j, e[j], eref)
        assert abs(w[j] - om.discarded) <= 1e-4 * om.discarded + 1e-10, (j, w[j], om.discarded)
    assert compared >= 4 and truncated >= 1, (compared, truncated)
