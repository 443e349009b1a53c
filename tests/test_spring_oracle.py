"""Pins of the SPRING oracle (Methods, "Variational Monte Carlo", eq. spring)
against facts of linear algebra that do not use its formula: the
parameter-space form of damped natural gradient, the minimum-norm solution
as the damping vanishes, the momentum fixed point, and invariance under a
shift of every gradient row (only the centred rows enter)."""
import numpy as np

from oracle import spring_oracle as S


def _case(N=12, P=40, seed=0):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((N, P)) * rng.uniform(0.1, 3.0, size=P)
    e = rng.standard_normal(N) * 2.0 - 50.0
    d0 = rng.standard_normal(P) * 0.1
    return O, e, d0


def test_sample_space_form_equals_parameter_space_form():
    """Obar^T (Obar Obar^T + l I)^-1 = (Obar^T Obar + l I)^-1 Obar^T (push-through
    identity): with eta = 0 the update is the damped natural-gradient step
    (S + l I)^-1 Obar^T eps with S = Obar^T Obar, a P x P solve."""
    O, e, _ = _case()
    lam = 1e-2
    d, _, _ = S.spring_update(O, e, None, 0.0, lam)
    Ob = O - O.mean(0)
    eps = e - e.mean()
    ref = np.linalg.solve(Ob.T @ Ob + lam * np.eye(O.shape[1]), Ob.T @ eps)
    np.testing.assert_allclose(d, ref, rtol=1e-9, atol=1e-11)


def test_vanishing_damping_gives_the_minimum_norm_solution():
    """lambda -> 0 with P > N: delta solves Obar delta = eps (eps is centred, so
    it lies in the range of the rank N-1 centred matrix) with the least norm,
    i.e. the pseudo-inverse solution."""
    O, e, _ = _case(N=10, P=30, seed=1)
    d, _, _ = S.spring_update(O, e, None, 0.0, 1e-10)
    Ob = O - O.mean(0)
    eps = e - e.mean()
    np.testing.assert_allclose(Ob @ d, eps, rtol=0, atol=1e-6)
    np.testing.assert_allclose(d, np.linalg.pinv(Ob) @ eps, rtol=1e-6, atol=1e-8)


def test_momentum_fixed_point():
    """eps = eta Obar delta_prev leaves only the momentum term: delta = eta delta_prev."""
    O, _, d0 = _case(seed=2)
    eta = 0.99
    Ob = O - O.mean(0)
    e = eta * (Ob @ d0) + 7.0          # any constant shift vanishes when centred
    d, _, _ = S.spring_update(O, e, d0, eta, 1e-3)
    np.testing.assert_allclose(d, eta * d0, rtol=0, atol=1e-12)


def test_shift_of_every_row_changes_nothing():
    O, e, d0 = _case(seed=3)
    a, Ka, _ = S.spring_update(O, e, d0, 0.9, 1e-3)
    b, Kb, _ = S.spring_update(O + np.linspace(-5, 5, O.shape[1]), e + 3.0, d0, 0.9, 1e-3)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(Ka, Kb, rtol=1e-9, atol=1e-9)
