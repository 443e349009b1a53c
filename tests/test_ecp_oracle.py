"""Pins of the non-local pseudopotential oracle (oracle/ecp_oracle.py): the
quadrature rules integrate the Legendre polynomials exactly up to their
degree, the rotations are uniform proper rotations, and for a wave function
that is spherical around the pseudopotential nucleus every ratio is 1, so
only the l = 0 channel survives: V_nl = v_0(|r - R|), a closed form."""
import math

import numpy as np
import pytest

from oracle import ecp_oracle as E
from recipes import hydrogen_like, two_electron_product


@pytest.mark.parametrize("nq,degree", [(4, 2), (6, 3), (12, 5)])
def test_quadrature_integrates_polynomials_of_its_degree(nq, degree):
    d, w = E.quadrature(nq)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    rng = np.random.default_rng(nq)
    for _ in range(20):
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b = rng.standard_normal(3)
        b /= np.linalg.norm(b)
        R = E.rotation(77, int(rng.integers(1000)), int(rng.integers(50)))
        dd = d @ R.T
        x = dd @ a
        # sphere averages: <1> = 1, <P_1> = <P_2> = 0, <(n.a)(n.b)> = a.b / 3
        assert abs((w * E.legendre(1, x)).sum()) < 1e-14
        assert abs((w * E.legendre(2, x)).sum()) < 1e-14
        assert abs((w * x * (dd @ b)).sum() - a @ b / 3) < 1e-14
        if degree >= 3:
            assert abs((w * x ** 3).sum()) < 1e-14
        if degree >= 4:
            assert abs((w * x ** 4).sum() - 1 / 5) < 1e-14     # <x^4> on the sphere = 1/5


def test_rotations_are_uniform_proper_rotations():
    Rs = np.stack([E.rotation(5, w, k) for w in range(200) for k in range(10)])
    for R in Rs[:50]:
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
    # a uniform (Haar) rotation has E[R] = 0 and E[R_ij^2] = 1/3
    se = 1.0 / math.sqrt(len(Rs))
    assert np.all(np.abs(Rs.mean(0)) < 5 * 0.58 * se)
    assert np.all(np.abs((Rs ** 2).mean(0) - 1 / 3) < 5 * 0.3 * se)


def _ecp(nq, terms, r_cut):
    return {"n_quad": nq, "r_cut": r_cut, "terms": terms}


@pytest.mark.parametrize("nq", [4, 6, 12])
def test_spherical_wave_function_keeps_only_the_s_channel(nq):
    """Psi = exp(-r) around the one nucleus: ratio 1 for every quadrature
    point, so V_nl = v_0(r) + 3 v_1(r) <P_1> + 5 v_2(r) <P_2> = v_0(r)."""
    system, arch, p = hydrogen_like(1.0, 1.0)
    terms = [[(3.0, 0, 1.5), (-1.0, 2, 0.7)], [(5.0, 1, 2.0)], [(2.0, 0, 0.9)]]
    r = np.random.default_rng(nq).standard_normal((16, 1, 3))
    r[0, 0] = [4.0, 0.0, 0.0]                     # beyond r_cut: no contribution
    V = E.nonlocal_energy(system, arch, p, r, [_ecp(nq, terms, 3.0)], seed=11)
    rad = np.linalg.norm(r[:, 0], axis=-1)
    want = np.where(rad < 3.0, 3.0 * np.exp(-1.5 * rad ** 2) - rad ** 2 * np.exp(-0.7 * rad ** 2), 0.0)
    np.testing.assert_allclose(V, want, rtol=0, atol=1e-12)


def test_two_electron_product_sums_over_electrons():
    """Psi = exp(-s0 r0 - s1 r1): both electrons see the s channel alone."""
    system, arch, p = two_electron_product()
    terms = [[(2.0, 0, 1.0)]]
    r = np.random.default_rng(3).standard_normal((8, 2, 3)) * 0.8
    V = E.nonlocal_energy(system, arch, p, r, [_ecp(4, terms, 2.5)], seed=2)
    rad = np.linalg.norm(r, axis=-1)
    want = (np.where(rad < 2.5, 2.0 * np.exp(-rad ** 2), 0.0)).sum(-1)
    np.testing.assert_allclose(V, want, rtol=0, atol=1e-12)
