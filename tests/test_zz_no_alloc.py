"""The allocation-free energy entry point agrees with the workspace entry point.

Some callers cannot call cudaMalloc (a framework that has reserved the whole
device budget, or a loop that must never enter the allocator); for them the
library evaluates energies in its own static device scratch. These tests call
it through the C ABI twice in a row and compare with the workspace entry point
in every arithmetic form, at the 40-qubit chi = 128 benchmark size as well,
check that neither PyTorch's allocator nor the device's free memory moves
across the calls, and that a term set too large for the scratch is rejected
with TNMPS_ERR_NOMEM. Collected last, so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest

from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

TOL = {"c128": 1e-12, "c64": 1e-6, "c64_bf16split": 1e-6}


def alloc_count():
    return torch.cuda.memory_stats().get("allocation.all.allocated", 0)


def check_against_workspace(m, terms, n, B, tol):
    ps = tnmps.PauliSum(n, terms)
    T = len(terms)
    e_ws = torch.zeros(B, dtype=torch.float64, device="cuda")
    pt_ws = torch.zeros((B, T), dtype=torch.float64, device="cuda")
    m.expect_dev(ps, e_ws, pt_ws)
    scale = sum(abs(t[0]) for t in terms)
    outs = [(torch.full((B,), float("nan"), dtype=torch.float64, device="cuda"),
             torch.full((B, T), float("nan"), dtype=torch.float64, device="cuda"))
            for _ in range(3)]
    m.expect_noalloc(ps, *outs[0])        # sets the scratch up on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = alloc_count()
    for e_na, pt_na in outs[1:]:          # two calls in a row
        m.expect_noalloc(ps, e_na, pt_na)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert alloc_count() == n0
    m.check()
    for e_na, pt_na in outs:
        assert np.allclose(e_na.cpu().numpy(), e_ws.cpu().numpy(), rtol=0, atol=tol * scale)
        assert np.allclose(pt_na.cpu().numpy(), pt_ws.cpu().numpy(), rtol=0, atol=tol)
    # energies alone (no per-term output: the scratch holds that region)
    e_only = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    m.expect_noalloc(ps, e_only)
    torch.cuda.synchronize()
    assert np.allclose(e_only.cpu().numpy(), e_ws.cpu().numpy(), rtol=0, atol=tol * scale)


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_bf16split"])
def test_noalloc_matches_workspace_entry_point(dtype):
    wl = inputs.workload("heis40")
    B = 4
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], B, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.apply_circuit(wl["circuit"], wl["thetas"][:B])
    check_against_workspace(m, wl["terms"], wl["n"], B, TOL[dtype])


@pytest.mark.parametrize("dtype", ["c64", "c64_bf16split"])
def test_noalloc_chi128_state(dtype):
    """One state of the chi = 128 benchmark workload (middle bonds at 128)
    with its Heisenberg chain; then the 2000 random strings, whose widest trie
    level does not fit the scratch for one state: TNMPS_ERR_NOMEM."""
    wl = inputs.workload("chi128")
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], 1, dtype=dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    m.apply_circuit(wl["circuit"], wl["thetas"][:1])
    assert m.bond_dims().max() == 128
    check_against_workspace(m, wl["terms"], wl["n"], 1, TOL[dtype])
    big = tnmps.PauliSum(wl["n"], wl["terms_random"])
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tnmps.TnmpsError) as ei:
        m.expect_noalloc(big, e)
    assert ei.value.status == 2 and "scratch" in str(ei.value)
    m.check()
