"""GPU parity of measurement sampling: the CUDA sampler against the oracle's
(same uniforms, same decision rule), closed forms and the Born rule."""
import numpy as np
import pytest

from oracle import mps as OM
from oracle import sampling as S
from oracle import statevector as SV
from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402

# outcomes decided by |u - P(0|...)| below these margins may differ by rounding
MARGIN = {"c128": 1e-9, "c64": 1e-4, "c64_bf16split": 1e-4}


def gpu_bits(n, chi, eps, circ, th, u, dtype):
    B = th.shape[0] if th is not None else 1
    m = tnmps.MPSBatch(n, chi, B, dtype=dtype, max_params=th.shape[1] if th is not None else 0,
                       eps=eps)
    m.apply_circuit(circ, th)
    return m, m.sample(u)


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_bf16split"])
def test_hea8_against_oracle(dtype):
    wl = inputs.workload("hea8", 1)
    th = wl["thetas"][:4]
    u = np.random.default_rng(8).random((4, 300, wl["n"]))
    _, bits = gpu_bits(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, u, dtype)
    for b in range(4):
        om = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], th[b])
        ref, margin = S.sample_mps(om, u[b])
        ok = margin > MARGIN[dtype]
        assert ok.mean() > 0.95
        assert np.array_equal(bits[b][ok], ref[ok])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_heis40_against_oracle(dtype):
    wl = inputs.workload("heis40")
    th = wl["thetas"][:2]
    u = np.random.default_rng(40).random((2, 128, wl["n"]))
    _, bits = gpu_bits(wl["n"], wl["chi_max"], wl["eps"], wl["circuit"], th, u, dtype)
    for b in range(2):
        om = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], th[b])
        ref, margin = S.sample_mps(om, u[b])
        ok = margin > MARGIN[dtype]
        assert ok.mean() > 0.9
        assert np.array_equal(bits[b][ok], ref[ok])


def test_ghz40_all_equal():
    n = 40
    circ = [("H", 0, -1, -1, 0.0, 1.0)] + [("CNOT", q, q + 1, -1, 0.0, 1.0) for q in range(n - 1)]
    u = np.random.default_rng(1).random((1, 500, n))
    _, bits = gpu_bits(n, 8, 1e-10, circ, None, u, "c64")
    expect = (u[0, :, n - 1] >= 0.5).astype(np.uint8)
    assert np.array_equal(bits[0], np.repeat(expect[:, None], n, axis=1))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_product_state_closed_form(dtype):
    n = 40
    rng = np.random.default_rng(2)
    th = rng.uniform(-np.pi, np.pi, (3, n))
    circ = [("RY", q, -1, q, 0.0, 1.0) for q in range(n)]
    u = rng.random((3, 400, n))
    _, bits = gpu_bits(n, 4, 1e-10, circ, th, u, dtype)
    p0 = np.cos(th / 2) ** 2
    expect = (u >= p0[:, None, :]).astype(np.uint8)
    ok = np.abs(u - p0[:, None, :]) > MARGIN[dtype]
    assert np.array_equal(bits[ok], expect[ok])


def test_born_rule_histogram():
    n = 5
    rng = np.random.default_rng(6)
    circ, P = inputs.hea_circuit(n, 3, ("RY", "RZ"))
    th = rng.uniform(-np.pi, np.pi, (1, P))
    _, bits = gpu_bits(n, 8, 1e-12, circ, th, rng.random((1, 40000, n)), "c64")
    idx = (bits[0].astype(np.int64) << np.arange(n)).sum(axis=1)
    freq = np.bincount(idx, minlength=1 << n) / idx.size
    psi = SV.run_circuit(n, circ, th[0])
    assert 0.5 * np.abs(freq - np.abs(psi) ** 2).sum() < 0.02


def test_bad_arguments():
    m = tnmps.MPSBatch(4, 4, 1, dtype="c64")
    u = torch.zeros((1, 0, 4), dtype=torch.float64, device="cuda")
    bits = torch.zeros((1, 0, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(tnmps.TnmpsError):
        m.sample_dev(u, bits)
