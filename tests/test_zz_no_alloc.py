"""The allocation-free energy entry point (for callers that cannot call
cudaMalloc) agrees with the workspace entry point, through the C ABI, on two
calls in a row. Collected last so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest

from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-6)])
def test_noalloc_matches_workspace_entry_point(dtype, tol):
    wl = inputs.workload("heis40")
    B = 4
    th = wl["thetas"][:B]
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], B, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.apply_circuit(wl["circuit"], th)
    ps = tnmps.PauliSum(wl["n"], wl["terms"])
    T = len(wl["terms"])
    e_ws = torch.zeros(B, dtype=torch.float64, device="cuda")
    pt_ws = torch.zeros((B, T), dtype=torch.float64, device="cuda")
    m.expect_dev(ps, e_ws, pt_ws)
    scale = sum(abs(t[0]) for t in wl["terms"])
    for _ in range(2):
        e_na = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
        pt_na = torch.full((B, T), float("nan"), dtype=torch.float64, device="cuda")
        m.expect_noalloc(ps, e_na, pt_na)
        torch.cuda.synchronize()
        m.check()
        assert np.allclose(e_na.cpu().numpy(), e_ws.cpu().numpy(), rtol=0, atol=tol * scale)
        assert np.allclose(pt_na.cpu().numpy(), pt_ws.cpu().numpy(), rtol=0, atol=tol)
