"""The tcgen05 matrix product on its own, against a float32 product of the
same bf16-rounded operands (a library routine, not the CUDA path)."""
import pytest
import torch

from paper_2504_06087_gb300 import fire

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 180, 256), (1000, 272, 256), (77, 16, 128),
                                   (4096, 192, 512)])
def test_tc_gemm_matches_float32_product(M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = fire.tc_gemm_selftest(A, Bt)
    ref = A.float() @ Bt.float().T
    err = (C - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * (K / 64) ** 0.5, (err, scale)
