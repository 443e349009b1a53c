"""Pins of the S+ swap-ratio oracle (oracle/spin_oracle.py) by closed forms of
two-electron product wave functions Psi = exp(-s0 |r_0| - s1 |r_1|)
(1 spin-up electron 0, 1 spin-down electron 1):
  swapping the two electrons gives Psi'/Psi = exp(-(s0 - s1)(|r_1| - |r_0|)),
  and for equal exponents the spatial part is symmetric (a singlet):
  every ratio is 1 and S+ Psi = 0, i.e. R_beta = 0."""
import numpy as np

from oracle import spin_oracle as SP
from recipes import two_electron_product


def test_swap_ratio_closed_form():
    s0, s1 = 1.6, 0.9
    system, arch, p = two_electron_product(s0=s0, s1=s1)
    r = np.random.default_rng(2).standard_normal((12, 2, 3))
    ratios, R = SP.swap_ratios(system, arch, p, r, beta=1)
    r0, r1 = np.linalg.norm(r[:, 0], axis=-1), np.linalg.norm(r[:, 1], axis=-1)
    want = np.exp(-(s0 - s1) * (r1 - r0))
    np.testing.assert_allclose(ratios[:, 0], want, rtol=1e-12)
    np.testing.assert_allclose(R, 1.0 - want, rtol=1e-12, atol=1e-12)


def test_singlet_has_no_s_plus_component():
    system, arch, p = two_electron_product(s0=1.2, s1=1.2)
    r = np.random.default_rng(3).standard_normal((12, 2, 3))
    ratios, R = SP.swap_ratios(system, arch, p, r, beta=1)
    np.testing.assert_allclose(ratios, 1.0, rtol=1e-12)
    np.testing.assert_allclose(R, 0.0, atol=1e-12)
