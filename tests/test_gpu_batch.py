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
