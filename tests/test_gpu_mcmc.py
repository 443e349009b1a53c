"""GPU parity of fire_mcmc_step against the full-recompute Metropolis oracle.

Decisions closer to the acceptance threshold than the rounding of the two
implementations (the oracle's margin |ln u - 2 ln ratio|) are not compared;
everything else (which moves were accepted, the final positions, log|Psi|)
must agree.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fire_oracle as O
from oracle import mcmc_oracle as M
from paper_2504_06087_gb300 import fire, synth
from recipes import hydrogen_like

pytestmark = pytest.mark.gpu


def _run(system, arch, p, prec, r_np, sigma, sweeps, seed, counter=0, refresh=32, k_cap=64, n_global=0,
         sigma_global=2.0):
    f = fire.Fire(system, arch, p, prec, k_cap=k_cap)
    r = torch.as_tensor(r_np, device=f.device).clone()
    out = f.mcmc_step(r, sigma, sweeps, refresh_every=refresh, seed=seed, counter=counter, n_global=n_global,
                      sigma_global=sigma_global)
    torch.cuda.synchronize()
    return f, r.cpu().numpy(), out


@pytest.mark.parametrize("sigma", [0.3, 1.0])
def test_water_fp64_decisions_match_oracle(sigma):
    w = synth.workload("water")
    r0, p = synth.make_inputs(w, 16)
    seed, counter = 1234567890123, 5
    f, r, out = _run(w.system, w.arch, p, "fp64", r0, sigma, 2, seed, counter, refresh=7)
    ref = M.mcmc_sweeps(w.system, w.arch, p, r0, sigma, 2, seed, counter)
    safe = ref["margin"] > 1e-8
    assert safe.sum() >= 12
    acc = out["accepted"].cpu().numpy()
    np.testing.assert_array_equal(acc[safe], ref["accepted"][safe])
    np.testing.assert_allclose(r[safe], ref["r"][safe], rtol=0, atol=1e-11)
    la = out["logabs"].cpu().numpy()
    np.testing.assert_allclose(la[safe], ref["logabs"][safe], rtol=1e-10, atol=1e-10)
    assert out["counter"] == counter + 2 * w.system.n_el
    assert out["n_accepted"] == int(acc.sum())
    assert 0 < out["n_accepted"] < 16 * 2 * w.system.n_el
    assert out["max_drift"] < 1e-9, out["max_drift"]


def test_fp64_woodbury_state_matches_rebuilds():
    """The same sweeps with the state rebuilt after every move and with the
    low-rank updates alone (one rebuild at the end) end in the same place."""
    w = synth.workload("water")
    r0, p = synth.make_inputs(w, 8)
    _, ra, oa = _run(w.system, w.arch, p, "fp64", r0, 0.5, 3, 77, refresh=1)
    _, rb, ob = _run(w.system, w.arch, p, "fp64", r0, 0.5, 3, 77, refresh=0)
    np.testing.assert_allclose(ra, rb, rtol=0, atol=1e-11)
    np.testing.assert_array_equal(oa["accepted"].cpu().numpy(), ob["accepted"].cpu().numpy())
    assert ob["max_drift"] < 1e-9, ob["max_drift"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hydrogen_mean_radius(prec):
    """|Psi|^2 = exp(-2r): <r> = 3/2 bohr within 4 standard errors."""
    system, arch, p = hydrogen_like(1.0, 1.0, width=32)
    W = 8192
    r0 = np.random.default_rng(5).standard_normal((W, 1, 3))
    _, r, out = _run(system, arch, p, prec, r0, 1.0, 150, 31)
    rad = np.linalg.norm(r[:, 0], axis=-1)
    se = math.sqrt(0.75 / W)
    assert abs(rad.mean() - 1.5) < 4 * se, (rad.mean(), se)
    assert 0.3 < out["n_accepted"] / (W * 150) < 0.9


def test_tiny_steps_are_accepted():
    w = synth.workload("water")
    r0, p = synth.make_inputs(w, 8)
    _, r, out = _run(w.system, w.arch, p, "fp64", r0, 1e-9, 1, 3)
    assert out["n_accepted"] == 8 * w.system.n_el
    np.testing.assert_allclose(r, r0, atol=1e-7)


@pytest.fixture(scope="module")
def c8h10_oracle():
    w = synth.workload("c8h10")
    r0, p = synth.make_inputs(w, 24)
    return w, r0, p, M.mcmc_sweeps(w.system, w.arch, p, r0, 0.3, 1, 2024)


def test_c8h10_fp64_low_rank_state_stays_exact(c8h10_oracle):
    """n_el = 58, float64 state, no rebuild inside the sweep: every decision
    equals the oracle's and the carried log|Psi| equals the rebuild at the
    end to float64 rounding -- including walkers where single determinants
    pass near their nodes (refactorised instead of Woodbury-updated)."""
    w, r0, p, ref = c8h10_oracle
    f, r, out = _run(w.system, w.arch, p, "fp64", r0, 0.3, 1, 2024, refresh=0)
    safe = ref["margin"] > 1e-8
    acc = out["accepted"].cpu().numpy()
    np.testing.assert_array_equal(acc[safe], ref["accepted"][safe])
    np.testing.assert_allclose(r[safe], ref["r"][safe], rtol=0, atol=1e-11)
    assert out["max_drift"] < 1e-8, out["max_drift"]


def test_c8h10_fp32_against_oracle_and_rebuild(c8h10_oracle):
    """n_el = 58, float32 state with float64 refreshes: decisions with a
    margin above the float32 rounding of ln|Psi'/Psi| equal the oracle's, the
    carried log|Psi| stays within float32 rounding of each rebuild, and the
    final log|Psi| matches the oracle at the final positions."""
    w, r0, p, ref = c8h10_oracle
    f, r, out = _run(w.system, w.arch, p, "fp32", r0, 0.3, 1, 2024, refresh=16)
    safe = ref["margin"] > 1e-3
    assert safe.sum() >= 12
    acc = out["accepted"].cpu().numpy()
    np.testing.assert_array_equal(acc[safe], ref["accepted"][safe])
    np.testing.assert_allclose(r[safe], ref["r"][safe], rtol=0, atol=1e-9)
    assert out["max_drift"] < 2e-3, out["max_drift"]
    la_ref, _ = O.logpsi_np(w.system, w.arch, p, r)
    la = out["logabs"].cpu().numpy()
    assert np.max(np.abs(la - la_ref) / np.maximum(np.abs(la_ref), 1.0)) < 1e-5


def test_c26h24_fp32_sweep_keeps_a_consistent_state():
    """n_el = 180 (the local-energy workload), 256 walkers, one sweep: the
    carried log|Psi| of every walker stays within 1e-2 of each float64
    rebuild (the conditioning test sends every determinant with
    kappa u w > 1e-4 to float64 ratios and refactorisation, so a run of 32
    moves accumulates at most ~32 x 1e-4 from the rest; over 4096 walkers
    the largest drift measured was 8.8e-3), and the final log|Psi| agrees
    with a separate fire_logpsi call at the final positions."""
    w = synth.workload("c26h24")
    r0, p = synth.make_inputs(w, 256)
    f, r, out = _run(w.system, w.arch, p, "fp32", r0, 0.3, 1, 99, refresh=32)
    assert out["max_drift"] < 1e-2, out["max_drift"]
    assert float(out["walker_drift"].max()) < 1e-2
    rate = out["n_accepted"] / (256 * w.system.n_el)
    assert 0.2 < rate < 0.99, rate
    g = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64)
    lp = g.logpsi(torch.as_tensor(r, device=g.device))["logabs"].cpu().numpy()
    np.testing.assert_allclose(out["logabs"].cpu().numpy(), lp, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------------------
# global single-electron jumps (Methods, "Improved Monte Carlo sampling")
# ---------------------------------------------------------------------------

def test_water_fp64_global_jumps_match_oracle():
    """Sweeps of 10 local moves and 6 global jumps (sigma_g = 2): every
    decision away from the threshold, the final positions and log|Psi| equal
    the full-recompute oracle with the same mixture proposals and Hastings
    factors."""
    w = synth.workload("water")
    r0, p = synth.make_inputs(w, 16)
    seed, counter, G = 987654321, 40, 6
    f, r, out = _run(w.system, w.arch, p, "fp64", r0, 0.3, 2, seed, counter, refresh=9, n_global=G)
    ref = M.mcmc_sweeps(w.system, w.arch, p, r0, 0.3, 2, seed, counter, n_global=G, sigma_global=2.0)
    safe = ref["margin"] > 1e-8
    assert safe.sum() >= 12
    acc = out["accepted"].cpu().numpy()
    np.testing.assert_array_equal(acc[safe], ref["accepted"][safe])
    np.testing.assert_allclose(r[safe], ref["r"][safe], rtol=0, atol=1e-11)
    la = out["logabs"].cpu().numpy()
    np.testing.assert_allclose(la[safe], ref["logabs"][safe], rtol=1e-10, atol=1e-10)
    assert out["counter"] == counter + 2 * (w.system.n_el + G)
    assert out["max_drift"] < 1e-9, out["max_drift"]
    # some global jumps were accepted: a walker moved an electron by more than
    # any local step could (8 sigma)
    assert np.max(np.abs(r - r0)) > 2.4


def test_c8h10_fp64_global_jumps_match_oracle():
    """n_el = 58 with 20 global jumps per sweep, float64 state, no rebuild
    inside the sweep: the jumps' update sets span two neighbourhoods."""
    w = synth.workload("c8h10")
    r0, p = synth.make_inputs(w, 12)
    ref = M.mcmc_sweeps(w.system, w.arch, p, r0, 0.3, 1, 555, n_global=20, sigma_global=2.0)
    f, r, out = _run(w.system, w.arch, p, "fp64", r0, 0.3, 1, 555, refresh=0, n_global=20)
    safe = ref["margin"] > 1e-8
    acc = out["accepted"].cpu().numpy()
    np.testing.assert_array_equal(acc[safe], ref["accepted"][safe])
    np.testing.assert_allclose(r[safe], ref["r"][safe], rtol=0, atol=1e-11)
    assert out["max_drift"] < 1e-8, out["max_drift"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hydrogen_mean_radius_from_global_jumps_alone(prec):
    """Local steps of 1e-9 bohr, two global jumps per sweep: the independence
    sampler with the Hastings factor samples exp(-2r), <r> = 3/2 (without
    the factor it would sample exp(-2r) rho(r), <r> = 1.25)."""
    system, arch, p = hydrogen_like(1.0, 1.0, width=32)
    W = 8192
    r0 = np.random.default_rng(6).standard_normal((W, 1, 3))
    _, r, out = _run(system, arch, p, prec, r0, 1e-9, 60, 17, n_global=2)
    rad = np.linalg.norm(r[:, 0], axis=-1)
    se = math.sqrt(0.75 / W)
    assert abs(rad.mean() - 1.5) < 4 * se, (rad.mean(), se)
