"""Plain FP64 CPU oracle of the S+ swap ratios.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.

What it computes (Supplementary "Low-rank updates in S+ operator"; Methods
"Low-rank wave function updates": for S+ the configurations differ in two
electrons): for a spin-down electron beta, the ratios
Psi(pi_{alpha beta} r) / Psi(r) for every spin-up electron alpha, where
pi_{alpha beta} swaps the positions of electrons alpha and beta (each keeps
its spin), and

    R_beta(r) = 1 - sum_alpha Psi(pi_{alpha beta} r) / Psi(r).

Every ratio is a full recompute of log|Psi| and sign with the dense oracle.
Reading P1: the sum runs over the n_up spin-up electrons (the printed bound
of the sum is garbled); beta is chosen by the caller.
"""
from __future__ import annotations

import numpy as np

from . import fire_oracle as O


def swap_ratios(system, arch, params, r_np: np.ndarray, beta: int):
    """(ratios [W, n_up], R_beta [W]) for the spin-down electron beta."""
    r = np.asarray(r_np, dtype=np.float64)
    nu = system.n_up
    lp, sg = O.logpsi_np(system, arch, params, r)
    out = np.zeros((r.shape[0], nu))
    for a in range(nu):
        q = r.copy()
        q[:, [a, beta]] = r[:, [beta, a]]
        lq, sq = O.logpsi_np(system, arch, params, q)
        out[:, a] = sq * sg * np.exp(lq - lp)
    return out, 1.0 - out.sum(axis=1)
