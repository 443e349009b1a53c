"""fire_local_energy_static: the local energy for callers that cannot
allocate device memory (see include/fire.h).

It must give the same result as fire_local_energy with a caller-allocated
workspace, call after call (the library-owned scratch keeps the previous
call's contents), and reject problems larger than its fixed scratch before
launching anything.  This file is collected last so that a run stopping at
the first failure has already run every other test; it also passes alone in
a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2504_06087_gb300 import fire, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def test_static_workspace_entry_matches_allocating_entry_twice():
    w = synth.workload("water")
    f = fire.Fire(w.system, w.arch, synth.init_params(w.system, w.arch, 1), "fp64")
    for call, seed in enumerate((1001, 2002)):
        r = synth.walkers(w.system, 12, seed)
        ref = f.local_energy(r)
        got = f.local_energy_static(r)
        torch.cuda.synchronize()
        assert got["status"] == 0, call
        np.testing.assert_array_equal(got["sign"].cpu().numpy(), ref["sign"].cpu().numpy())
        for k in ("e_loc", "logabs", "e_kin", "e_pot"):
            assert rel(got[k].cpu().numpy(), ref[k].cpu().numpy()).max() < 1e-10, (call, k)


def test_static_workspace_entry_rejects_problems_beyond_its_size():
    w = synth.workload("c8h10")
    f = fire.Fire(w.system, w.arch, synth.init_params(w.system, w.arch, 2), "fp32")
    r = synth.walkers(w.system, 64, 3003)
    out = f.local_energy_static(r, check=False)
    assert out["status"] == 8       # FIRE_ERR_WORKSPACE, detected on the host
    assert b"static workspace holds" in fire.lib().fire_last_error()
