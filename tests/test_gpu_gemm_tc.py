"""Parity of the tcgen05 BF16 GEMM (C = A B^T, FP32 accumulate) against a
float64 matmul of the same BF16-rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import tnmps  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 128, 320), (300, 256, 256),
                                   (1000, 320, 4096), (7, 5, 8), (256, 1, 64)])
def test_gemm_bf16_matches_fp64(M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 13 + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    c = tnmps.gemm_bf16(a.cuda(), b.cuda())
    torch.cuda.synchronize()
    ref = a.double() @ b.double().T
    # exact BF16 products, FP32 accumulation of K terms: error <= K u32 sum|ab|
    bound = K * 2.0 ** -24 * (a.double().abs() @ b.double().abs().T) + 1e-30
    assert torch.all((c.double().cpu() - ref).abs() <= 2 * bound)
