"""The tcgen05 matrix product on its own, against a float32 product of the
same bf16-rounded operands (a library routine, not the CUDA path)."""
import pytest
import torch

from paper_2504_06087_gb300 import fire

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 180, 256), (1000, 272, 256), (77, 16, 128),
                                   (4096, 192, 512), (40000, 180, 256), (20011, 256, 128)])
def test_tc_gemm_matches_float32_product(M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = fire.tc_gemm_selftest(A, Bt)
    ref = A.float() @ Bt.float().T
    err = (C - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * (K / 64) ** 0.5, (err, scale)


@pytest.mark.parametrize("nc,tol,M", [(1, 1e-2, 640), (2, 5e-5, 640), (3, 5e-6, 640), (3, 5e-6, 30001),
                                      (2, 5e-5, 30001)])
def test_split_bf16_product_reaches_its_precision(nc, tol, M):
    """x = x0 + x1 (+ x2) in bf16 components; the 1 / 3 / 6 component
    products approach the float32 product of the unsplit values (the large M
    gives every CTA of the persistent grid several tiles)."""
    g = torch.Generator(device="cpu").manual_seed(7 + nc)
    N, K = 200, 256
    A = torch.randn(M, K, generator=g, dtype=torch.float32).cuda()
    B = torch.randn(N, K, generator=g, dtype=torch.float32).cuda()
    C = fire.tc_gemm_selftest(fire.split_bf16(A, nc), fire.split_bf16(B, nc), nc)
    ref = (A.double() @ B.double().T)
    err = ((C.double() - ref).abs().max() / ref.abs().max()).item()
    assert err < tol, err
