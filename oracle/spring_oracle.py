"""Plain FP64 CPU oracle of the SPRING parameter update.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.

What it computes (Methods, "Variational Monte Carlo", eq. spring): for a batch
of N samples with per-sample log-derivative rows O_i = d ln|Psi(r_i)| / d theta
(i = 1..N, P parameters) and local energies E_L(r_i),

    Obar_i = O_i - (1/N) sum_j O_j,        eps_i = E_L(r_i) - (1/N) sum_j E_L(r_j),
    delta  = Obar^T (Obar Obar^T + lambda I)^-1 (eps - eta Obar delta_prev) + eta delta_prev.

Reading S1 (the printed equation): the paper writes the update with the
centred matrix as P x N (columns = samples), Obar (Obar^T Obar + lambda I)^-1
(eps - Obar eta delta_prev); the N-vector eps - Obar eta delta_prev only has
consistent dimensions with the transposed product in the second term.  With
Obar stored as N x P (rows = samples, the layout of the per-walker gradient
rows) the update above is the same formula: an N x N Gram matrix, a damped
N x N solve, and the parameter-space vector Obar^T x plus the momentum term.
No 1/N normalisation is applied beyond the printed one.

Every step is the plain definition in float64: numpy means, a matrix
product for the Gram matrix, numpy.linalg.solve for the damped system.
"""
from __future__ import annotations

import numpy as np


def spring_update(O, e_loc, delta_prev, eta: float, lam: float):
    """(delta [P], Gram [N, N], x [N]) of one SPRING step, all float64."""
    O = np.asarray(O, dtype=np.float64)
    e = np.asarray(e_loc, dtype=np.float64)
    Ob = O - O.mean(axis=0, keepdims=True)
    eps = e - e.mean()
    d0 = np.zeros(O.shape[1]) if delta_prev is None else np.asarray(delta_prev, dtype=np.float64)
    K = Ob @ Ob.T
    rhs = eps - eta * (Ob @ d0)
    x = np.linalg.solve(K + lam * np.eye(K.shape[0]), rhs)
    return Ob.T @ x + eta * d0, K, x
