"""Pins of the Metropolis oracle (single-electron moves, full recompute).

Each pin checks the sampler against something other than itself: published
known-answer vectors of the generator, the moments of the normal
distribution, a closed-form wave function whose acceptance decisions can be
written out by hand, and the exact mean radius of the hydrogen ground state
sampled from |Psi|^2.
"""
import math
import os

import numpy as np
import pytest

from oracle import fire_oracle as O
from oracle import mcmc_oracle as M
from paper_2504_06087_gb300 import synth
from recipes import hydrogen_like, two_electron_product

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) >= 2
    for row in rows:
        v = [int(x, 16) for x in row]
        out = M.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniforms_stay_inside_the_open_interval():
    assert 0.0 < M.u01(0) < 1e-9
    assert 1.0 - 1e-9 < M.u01(0xFFFFFFFF) < 1.0


def test_proposals_are_standard_normal():
    """Box-Muller output: zero mean, unit variance, uncorrelated components,
    95 % of the mass inside +-1.96 (so a wrong radius or angle fails)."""
    N = 400_000
    xi, u = M.proposal(2024, 3, np.arange(N))
    se = 1.0 / math.sqrt(N)
    assert np.all(np.abs(xi.mean(0)) < 5 * se)
    assert np.all(np.abs(xi.var(0) - 1.0) < 5 * math.sqrt(2.0) * se)
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 * se)
    inside = (np.abs(xi) < 1.959963984540054).mean(0)
    assert np.all(np.abs(inside - 0.95) < 5 * math.sqrt(0.95 * 0.05) * se)
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12) * se
    # streams differ by walker and by move
    xi2, _ = M.proposal(2024, 4, np.arange(8))
    assert not np.allclose(xi[:8], xi2)


def test_decisions_follow_the_closed_form_ratio():
    """Psi = exp(-s0 |r_0| - s1 |r_1|): the accept decisions of the oracle
    sweep equal ln u < 2 (ln|Psi'| - ln|Psi|) written from the closed form."""
    s0, s1 = 1.6, 0.9
    system, arch, p = two_electron_product(s0=s0, s1=s1)
    r0 = np.random.default_rng(7).standard_normal((64, 2, 3))
    sigma, seed = 0.8, 99
    out = M.mcmc_sweeps(system, arch, p, r0, sigma, 3, seed, counter=11)
    r = r0.copy()
    acc = np.zeros(64, dtype=np.int64)
    s = np.array([s0, s1])
    for sweep in range(3):
        for k in range(2):
            xi, u = M.proposal(seed, 11 + sweep * 2 + k, np.arange(64))
            rn = r[:, k] + sigma * xi
            dl = -s[k] * (np.linalg.norm(rn, axis=-1) - np.linalg.norm(r[:, k], axis=-1))
            ok = np.log(u) < 2 * dl
            r[ok, k] = rn[ok]
            acc += ok
    safe = out["margin"] > 1e-9
    assert safe.sum() > 50
    np.testing.assert_array_equal(out["accepted"][safe], acc[safe])
    np.testing.assert_allclose(out["r"][safe], r[safe], rtol=0, atol=1e-13)
    assert 0 < acc.sum() < 64 * 6
    assert out["counter"] == 11 + 3 * 2


def test_hydrogen_mean_radius():
    """|Psi|^2 = exp(-2r): <r> = 3/2 bohr; the walkers after burn-in are
    independent samples, so the batch mean must lie within 4 standard errors.
    A rule accepting with |Psi'/Psi| instead of its square would give 3."""
    system, arch, p = hydrogen_like(1.0, 1.0)
    W = 4000
    r0 = np.random.default_rng(5).standard_normal((W, 1, 3))
    out = M.mcmc_sweeps(system, arch, p, r0, 1.0, 120, 31)
    rad = np.linalg.norm(out["r"][:, 0], axis=-1)
    se = math.sqrt(0.75 / W)     # Var r = 3 / (4 sigma^2) for exp(-2 r)
    assert abs(rad.mean() - 1.5) < 4 * se, (rad.mean(), se)
    assert 0.3 < out["accepted"].mean() / 120 < 0.9
    # log|Psi| carried with the walkers is log|Psi| at the final positions
    la, _ = O.logpsi_np(system, arch, p, out["r"])
    np.testing.assert_allclose(out["logabs"], la, rtol=0, atol=1e-12)


def test_tiny_steps_are_accepted():
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 4)
    out = M.mcmc_sweeps(w.system, w.arch, p, r, 1e-9, 1, 5)
    assert np.all(out["accepted"] == w.system.n_el)
    np.testing.assert_allclose(out["r"], r, atol=1e-7)


# ---------------------------------------------------------------------------
# global single-electron jumps (Methods, "Improved Monte Carlo sampling")
# ---------------------------------------------------------------------------

def test_gmm_density_closed_form():
    """rho_global at a nucleus of a two-centre mixture, written out:
    (Z1 + Z2 exp(-D^2 / 2 s^2)) / (Z1 + Z2) (2 pi s^2)^(-3/2)."""
    R = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 4.0]])
    Z = np.array([6.0, 2.0])
    s = 2.0
    want = math.log((6.0 + 2.0 * math.exp(-25.0 / 8.0)) / 8.0 * (2 * math.pi * 4.0) ** -1.5)
    got = M.log_gmm_density(np.array([0.0, 0.0, 0.0]), R, Z, s)
    assert abs(float(got) - want) < 1e-13


def test_global_proposals_follow_the_mixture():
    """Mixture components drawn with probability Z_m / sum Z, displacements
    N(0, sigma_g^2 I) around the chosen nucleus; the moved electron is
    uniform over the electrons."""
    R = np.array([[0.0, 0.0, 0.0], [40.0, 0.0, 0.0], [0.0, 60.0, 0.0]])
    Z = np.array([8.0, 1.0, 1.0])
    N, s = 300_000, 2.0
    rp, u = M.global_proposal(77, 12, np.arange(N), R, Z, s)
    comp = np.argmin(((rp[:, None, :] - R) ** 2).sum(-1), axis=1)     # nuclei 40+ bohr apart
    se = 1.0 / math.sqrt(N)
    for m in range(3):
        pm = Z[m] / Z.sum()
        assert abs((comp == m).mean() - pm) < 5 * math.sqrt(pm * (1 - pm)) * se
        d = (rp[comp == m] - R[m]) / s
        assert np.all(np.abs(d.mean(0)) < 0.05) and np.all(np.abs(d.var(0) - 1.0) < 0.05)
    ks = np.array([M.global_electron(5, mv, 7) for mv in range(7000)])
    counts = np.bincount(ks, minlength=7)
    assert counts.min() > 850 and counts.max() < 1150


def test_global_decisions_follow_the_closed_form_ratio():
    """Psi = exp(-s0 |r_0| - s1 |r_1|) on one nucleus at the origin:
    accept iff ln u < 2 (ln|Psi'| - ln|Psi|) + (|r'_k|^2 - |r_k|^2) / (2 sigma_g^2),
    the Hastings factor rho(r)/rho(r') of a single Gaussian written out."""
    s0, s1, sg = 1.6, 0.9, 2.0
    system, arch, p = two_electron_product(s0=s0, s1=s1)
    r0 = np.random.default_rng(8).standard_normal((64, 2, 3))
    sigma, seed, G = 0.7, 4242, 3
    out = M.mcmc_sweeps(system, arch, p, r0, sigma, 2, seed, counter=3, n_global=G, sigma_global=sg)
    r = r0.copy()
    acc = np.zeros(64, dtype=np.int64)
    s = np.array([s0, s1])
    for sweep in range(2):
        for j in range(2 + G):
            move = 3 + sweep * (2 + G) + j
            if j < 2:
                k = j
                xi, u = M.proposal(seed, move, np.arange(64))
                rn = r[:, k] + sigma * xi
                hast = 0.0
            else:
                k = M.global_electron(seed, move, 2)
                xi, u = M.proposal(seed, move, np.arange(64))
                rn = sg * xi                                   # the only component: the origin
                hast = ((rn ** 2).sum(-1) - (r[:, k] ** 2).sum(-1)) / (2 * sg ** 2)
            dl = -s[k] * (np.linalg.norm(rn, axis=-1) - np.linalg.norm(r[:, k], axis=-1))
            ok = np.log(u) < 2 * dl + hast
            r[ok, k] = rn[ok]
            acc += ok
    safe = out["margin"] > 1e-9
    assert safe.sum() > 50
    np.testing.assert_array_equal(out["accepted"][safe], acc[safe])
    np.testing.assert_allclose(out["r"][safe], r[safe], rtol=0, atol=1e-13)
    assert out["counter"] == 3 + 2 * (2 + G)


def test_hydrogen_mean_radius_from_global_moves_alone():
    """Global jumps only (local steps of 1e-9 bohr move nothing): the
    independence sampler with the Hastings factor rho(r)/rho(r') samples
    |Psi|^2 = exp(-2r), <r> = 3/2.  Without the factor the chain would sample
    exp(-2r) rho(r) instead (<r> = 1.25 for sigma_g = 2)."""
    system, arch, p = hydrogen_like(1.0, 1.0)
    W = 4000
    r0 = np.random.default_rng(6).standard_normal((W, 1, 3))
    out = M.mcmc_sweeps(system, arch, p, r0, 1e-9, 60, 17, n_global=2, sigma_global=2.0)
    rad = np.linalg.norm(out["r"][:, 0], axis=-1)
    se = math.sqrt(0.75 / W)
    assert abs(rad.mean() - 1.5) < 4 * se, (rad.mean(), se)
    moved = np.abs(out["r"] - r0).max(axis=(1, 2)) > 1e-6
    assert moved.mean() > 0.95
