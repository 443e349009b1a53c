"""The SIMT multiply-add probe computes the chains it claims (so its timing
counts real work): x <- a x + b for K rounds has the closed form
x_K = a^K x_0 + b (1 - a^K) / (1 - a)."""
import numpy as np
import pytest
import torch

from paper_2504_06087_gb300 import fire

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt,a,b,tol", [(torch.float64, 0.9999999, 1e-7, 1e-12), (torch.float32, 0.9999, 1e-4, 1e-4)])
def test_fma_probe_chains_follow_the_closed_form(dt, a, b, tol):
    blocks, iters = 3, 1000
    out = torch.empty(blocks * 256, dtype=dt, device="cuda")
    code = 0 if dt == torch.float64 else 1
    rc = fire.lib().fire_selftest_fma_rate(code, iters, blocks, out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0
    K = 4 * ((iters + 3) // 4)
    aK = a ** K
    x0 = (np.arange(blocks * 256) & 7).astype(np.float64)
    want = sum(aK * (x0 + j) + b * (1 - aK) / (1 - a) for j in range(8))
    got = out.double().cpu().numpy()
    assert np.max(np.abs(got - want) / np.abs(want)) < tol
