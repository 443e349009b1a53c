"""GPU parity of fire_spin_ratios (S+ swap ratios) with the full-recompute
oracle (oracle/spin_oracle.py).

Tolerances per ratio: FP64 state 1e-10 max(|ratio_ref|, 1); float32 state
1e-3 max(|ratio_ref|, 1), the float32 accuracy of a low-rank log-ratio that
the sampler's decisions are held to (measured 1.1e-4 on water).  R_beta = 1 - sum of the ratios to the same tolerance relative
to 1 + sum |ratio_ref|.  Closed forms: the two-electron product and its
singlet (R_beta = 0)."""
import numpy as np
import pytest

from oracle import spin_oracle as SP
from paper_2504_06087_gb300 import fire, synth
from recipes import two_electron_product

pytestmark = pytest.mark.gpu


def _check(out, ref_ratios, ref_r, tol):
    got = out["ratios"].cpu().numpy()
    assert np.all(np.abs(got - ref_ratios) <= tol * np.maximum(np.abs(ref_ratios), 1.0)), \
        np.max(np.abs(got - ref_ratios) / np.maximum(np.abs(ref_ratios), 1.0))
    scale = 1.0 + np.abs(ref_ratios).sum(1)
    assert np.all(np.abs(out["r_beta"].cpu().numpy() - ref_r) <= tol * scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_water_swap_ratios_match_oracle(prec, tol):
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 16)
    for beta in (5, 9):
        ref_ratios, ref_r = SP.swap_ratios(w.system, w.arch, p, r, beta)
        out = fire.Fire(w.system, w.arch, p, prec).spin_ratios(r, beta)
        _check(out, ref_ratios, ref_r, tol)


def test_c8h10_swap_ratios_match_oracle():
    """n_el = 58: swaps whose update sets span two neighbourhoods."""
    w = synth.workload("c8h10")
    r, p = synth.make_inputs(w, 4)
    ref_ratios, ref_r = SP.swap_ratios(w.system, w.arch, p, r, 40)
    out = fire.Fire(w.system, w.arch, p, "fp64").spin_ratios(r, 40)
    _check(out, ref_ratios, ref_r, 1e-10)


def test_singlet_closed_form_on_gpu():
    system, arch, p = two_electron_product(s0=1.2, s1=1.2)
    arch.width = arch.jastrow_width = 32
    p = two_electron_product_params(system, arch)
    r = np.random.default_rng(3).standard_normal((32, 2, 3))
    out = fire.Fire(system, arch, p, "fp64", k_cap=4).spin_ratios(r, 1)
    np.testing.assert_allclose(out["ratios"].cpu().numpy(), 1.0, rtol=1e-12)
    np.testing.assert_allclose(out["r_beta"].cpu().numpy(), 0.0, atol=1e-12)


def two_electron_product_params(system, arch):
    """The singlet recipe at the width the library takes (multiple of 32)."""
    from recipes import const_h_params
    p = const_h_params(system, arch)
    p["orb_w"][:] = 0.0
    p["orb_w"][0, 0, :, 0] = 1.0
    p["orb_w"][1, 0, :, 1] = 1.0
    p["env_pi"][:] = 0.0
    p["env_pi"][0, 0, 0, 0, :] = [1.0, 0.0]
    p["env_pi"][1, 0, 1, 0, :] = [0.0, 1.0]
    p["env_sigma"][0] = [1.2, 1.2]
    return p


def test_bad_beta_is_rejected():
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 2)
    f = fire.Fire(w.system, w.arch, p, "fp64")
    assert f.spin_ratios(r, 2, check=False)["status"] == 1      # a spin-up electron
    assert f.spin_ratios(r, 10, check=False)["status"] == 1
