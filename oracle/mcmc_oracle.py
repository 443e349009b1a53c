"""Plain FP64 CPU oracle of the Metropolis walker update (single-electron moves).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.

What it computes (Methods, "Improved Monte Carlo sampling"; Supplementary
"Hyperparameters": single-electron Gaussian moves): one sweep moves electron
k = 0, 1, ..., n-1 in turn.  For each k, every walker proposes
r'_k = r_k + sigma xi with xi ~ N(0, I_3) and accepts with probability
min(1, |Psi(r')/Psi(r)|^2).  Here every proposal is evaluated by a full
recompute of log|Psi(r')| with the dense oracle (no low-rank update); the
CUDA path must take the same decisions with its local recompute and
determinant-lemma ratios.

Random numbers (readings M1-M3, also listed in the design notes):
  M1  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = the 64-bit
      seed as (low word, high word), counter = (move low word, move high
      word, walker, stream); move = counter_in + sweep * n + k without
      global moves (M6 gives the numbering with them).
  M2  stream 0 gives four uniforms u_j = (x_j + 1/2) / 2^32 and, by the
      Box-Muller transform, xi = (a cos 2 pi u_1, a sin 2 pi u_1,
      b cos 2 pi u_3) with a = sqrt(-2 ln u_0), b = sqrt(-2 ln u_2).
  M3  stream 1 gives the acceptance uniform u = u_0; a move is accepted iff
      ln u < 2 (ln|Psi(r')| - ln|Psi(r)|) and the new value is finite.

Global single-electron jumps (Methods, "Improved Monte Carlo sampling": the
Gaussian-mixture proposal rho_global(r') = sum_m Z_m N(r' | R_m, sigma_g^2 I)
/ sum_m Z_m and its ratio correction rho(r)/rho(r'); Supplementary
"Hyperparameters": 20 global moves, sigma_g = 2):
  M6  a sweep is n local moves (k = 0 .. n-1) followed by G global moves;
      move = counter_in + sweep (n + G) + j for the j-th move of the sweep.
  M7  the electron of a global move is shared by all walkers:
      k = floor(n u) with u from the word 0 of counter (move low, move high,
      2^32 - 1, 2); per walker, the mixture component is the first m with
      u Z_tot < Z_1 + ... + Z_m (u from word 0 of stream 2), and
      r'_k = R_m + sigma_g xi with xi from stream 0 as in M2.
  M8  a global move is accepted iff
      ln u < 2 (ln|Psi(r')| - ln|Psi(r)|) + ln rho(r_k) - ln rho(r'_k).
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

from . import fire_oracle as O

MASK = 0xFFFFFFFF
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds (SC'11, section 5).  counter: four words,
    key: two words; each a Python int or a numpy array (broadcast together).
    Returns four numpy uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & np.uint64(MASK) for x in counter)
    k0, k1 = (np.asarray(x, dtype=np.uint64) & np.uint64(MASK) for x in key)
    m0, m1, mk = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1), np.uint64(MASK)
    s32 = np.uint64(32)
    for _ in range(10):
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> s32) ^ c1 ^ k0) & mk, p1 & mk, ((p0 >> s32) ^ c3 ^ k1) & mk, p0 & mk
        k0 = (k0 + np.uint64(PHILOX_W0)) & mk
        k1 = (k1 + np.uint64(PHILOX_W1)) & mk
    return c0, c1, c2, c3


def u01(x):
    """Uniform in (0, 1) from a 32-bit word: (x + 1/2) / 2^32."""
    return (np.asarray(x, dtype=np.float64) + 0.5) / 4294967296.0


def proposal(seed: int, move: int, walkers) -> Tuple[np.ndarray, np.ndarray]:
    """(xi [W, 3], acceptance uniforms u [W]) of the walkers' move (M1-M3)."""
    wk = np.asarray(walkers, dtype=np.uint64)
    key = (seed & MASK, (seed >> 32) & MASK)
    m_lo, m_hi = move & MASK, (move >> 32) & MASK
    a = philox4x32_10((m_lo, m_hi, wk, 0), key)
    b = philox4x32_10((m_lo, m_hi, wk, 1), key)
    ra = np.sqrt(-2.0 * np.log(u01(a[0])))
    rb = np.sqrt(-2.0 * np.log(u01(a[2])))
    t1 = 2.0 * math.pi * u01(a[1])
    t3 = 2.0 * math.pi * u01(a[3])
    xi = np.stack([ra * np.cos(t1), ra * np.sin(t1), rb * np.cos(t3)], axis=-1)
    return xi, u01(b[0])


def global_electron(seed: int, move: int, n: int) -> int:
    """Electron moved by the global jump `move`, the same for every walker (M7)."""
    key = (seed & MASK, (seed >> 32) & MASK)
    c = philox4x32_10((move & MASK, (move >> 32) & MASK, MASK, 2), key)
    return min(int(math.floor(float(u01(c[0])) * n)), n - 1)


def global_proposal(seed: int, move: int, walkers, nuc_pos, nuc_charge, sigma_g: float):
    """(r' [W, 3], acceptance uniforms u [W]) of a global jump (M7): a mixture
    component m with probability Z_m / sum Z, then r' = R_m + sigma_g xi."""
    wk = np.asarray(walkers, dtype=np.uint64)
    key = (seed & MASK, (seed >> 32) & MASK)
    m_lo, m_hi = move & MASK, (move >> 32) & MASK
    xi, u = proposal(seed, move, walkers)
    c = philox4x32_10((m_lo, m_hi, wk, 2), key)
    z = np.asarray(nuc_charge, dtype=np.float64)
    cum = np.cumsum(z)
    comp = np.searchsorted(cum, u01(c[0]) * cum[-1], side="right")
    comp = np.minimum(comp, z.size - 1)
    return np.asarray(nuc_pos, dtype=np.float64)[comp] + sigma_g * xi, u


def log_gmm_density(x, nuc_pos, nuc_charge, sigma_g: float) -> np.ndarray:
    """ln rho_global(x) for points x [..., 3] (Methods, the mixture proposal)."""
    R = np.asarray(nuc_pos, dtype=np.float64)
    z = np.asarray(nuc_charge, dtype=np.float64)
    d2 = ((np.asarray(x)[..., None, :] - R) ** 2).sum(-1)             # [..., N]
    e = np.log(z) - d2 / (2.0 * sigma_g ** 2)
    mx = e.max(-1, keepdims=True)
    return (mx[..., 0] + np.log(np.exp(e - mx).sum(-1)) - np.log(z.sum())
            - 1.5 * np.log(2.0 * math.pi * sigma_g ** 2))


def mcmc_sweeps(system, arch, params, r_np: np.ndarray, sigma: float, n_sweeps: int, seed: int,
                counter: int = 0, n_global: int = 0, sigma_global: float = 2.0) -> Dict[str, np.ndarray]:
    """n_sweeps sweeps of single-electron Metropolis moves, full recompute.

    Returns the final positions, log|Psi| and sign there, per-walker accepted
    counts, and per-walker smallest decision margin |ln u - 2 ln ratio|
    (decisions closer than rounding to the threshold may legitimately differ
    between two correct implementations)."""
    r = np.array(r_np, dtype=np.float64, copy=True)
    W, n = r.shape[0], r.shape[1]
    lp, sg = O.logpsi_np(system, arch, params, r)
    acc = np.zeros(W, dtype=np.int64)
    margin = np.full(W, np.inf)
    per = n + n_global
    for sweep in range(n_sweeps):
        for j in range(per):
            move = counter + sweep * per + j
            rp = r.copy()
            if j < n:
                k = j
                xi, u = proposal(seed, move, np.arange(W))
                rp[:, k] = r[:, k] + sigma * xi
                corr = np.zeros(W)
            else:
                k = global_electron(seed, move, n)
                rp[:, k], u = global_proposal(seed, move, np.arange(W), system.nuc_pos, system.nuc_charge,
                                              sigma_global)
                corr = (log_gmm_density(r[:, k], system.nuc_pos, system.nuc_charge, sigma_global)
                        - log_gmm_density(rp[:, k], system.nuc_pos, system.nuc_charge, sigma_global))
            lpn, sgn = O.logpsi_np(system, arch, params, rp)
            with np.errstate(invalid="ignore", over="ignore"):
                lr = lpn - lp
                ok = np.isfinite(lpn) & (np.log(u) < 2.0 * lr + corr)
                m = np.abs(np.log(u) - 2.0 * lr - corr)
            margin = np.minimum(margin, np.where(np.isfinite(m), m, np.inf))
            r[ok] = rp[ok]
            lp = np.where(ok, lpn, lp)
            sg = np.where(ok, sgn, sg)
            acc += ok
    return {"r": r, "logabs": lp, "sign": sg, "accepted": acc, "margin": margin,
            "counter": counter + n_sweeps * per}
