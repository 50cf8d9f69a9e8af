"""Failure detection without a GPU fault. Every device-side wait of the
tensor-core pipelines gives up after a bounded number of SM clocks, raises a
flag and lets its kernel return; the host reports the flag as
TNMPS_ERR_TIMEOUT and the context stays usable. Here a diagnostic kernel waits
on an mbarrier phase that nothing completes (nothing is in flight on it), so
the wait runs out after about a millisecond."""
import numpy as np
import pytest

from oracle import energy as OE
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

TIMEOUT = 8


def small_case():
    n = 6
    circ, P = inputs.hea_circuit(n, 2, ("RY", "RZ"))
    th = np.random.default_rng(1).uniform(-np.pi, np.pi, (2, P))
    terms = inputs.random_pauli_terms(n, 12, 3, np.random.default_rng(2))
    return n, circ, P, th, terms


@pytest.mark.parametrize("dtype", ["c128", "c64_bf16split"])
def test_wait_that_runs_out_is_reported_and_the_context_recovers(dtype):
    n, circ, P, th, terms = small_case()
    m = tnmps.MPSBatch(n, 8, 2, dtype=dtype, max_params=P, eps=1e-12)
    m.debug_wait_timeout(2_000_000)
    with pytest.raises(tnmps.TnmpsError) as ei:
        m.check()
    assert ei.value.status == TIMEOUT and "wait" in str(ei.value)
    m.reset()                               # clears the flag
    m.check()
    m.apply_circuit(circ, th)
    e = m.expect(tnmps.PauliSum(n, terms))
    tol = 1e-10 if dtype == "c128" else 1e-5
    for b in range(2):
        ref = OE.energy(n, circ, th[b], terms, "dense")
        assert abs(e[b] - ref) <= tol * sum(abs(t[0]) for t in terms)


def test_synchronising_call_reports_a_pending_timeout():
    n, circ, P, th, terms = small_case()
    m = tnmps.MPSBatch(n, 8, 2, dtype="c64", max_params=P, eps=1e-12)
    m.apply_circuit(circ, th)
    m.debug_wait_timeout(1_000_000)
    with pytest.raises(tnmps.TnmpsError) as ei:
        m.expect(tnmps.PauliSum(n, terms))     # host outputs: synchronises and checks
    assert ei.value.status == TIMEOUT


def test_wait_limit_is_checked_and_surrogate_check_passes():
    m = tnmps.MPSBatch(4, 4, 1, dtype="c64")
    for bad in (0, -5, (1 << 31) + 1):
        with pytest.raises(tnmps.TnmpsError) as ei:
            m.debug_wait_timeout(bad)
        assert ei.value.status == 1
    m.check()
    s = tnmps.Surrogate(16, 32, max_batch=64)
    s.set_params(np.random.default_rng(3).normal(size=s.n_params).astype(np.float32) * 0.1)
    y = s.forward(torch.randn(64, 16, device="cuda"))
    s.check()                                   # a GEMM that completed reports nothing
    assert bool(torch.all(torch.isfinite(y)))
