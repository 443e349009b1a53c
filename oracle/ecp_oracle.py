"""Plain FP64 CPU oracle of the non-local pseudopotential energy.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.

What it computes (Methods "Low-rank wave function updates": the non-local
pseudopotential needs ratios Psi(r')/Psi(r) of configurations that differ in
one electron; Supplementary "Effective core potential" and "Hyperparameters":
a per-species number of quadrature points, 4 for Li-Ne, 6 for Na-Ar, 12 for
K-Kr; Methods "Energy extrapolation": T_ecp = n_el N_quad T_upd).  The paper
uses the ccECP tables, which are not available here; the semi-local form is
the standard one with synthetic coefficients supplied by the caller:

    V_nl(r) = sum_k sum_l v_l(|r_k - R_m|) (2l + 1)
              sum_q w_q P_l(rhat_k . n_q) Psi(r_1 .. R_m + |r_k - R_m| n_q .. r_n) / Psi(r),
    v_l(x)  = sum_j c_lj x^p_lj exp(-a_lj x^2),

with m the pseudopotential nucleus of electron k, rhat_k the unit vector from
R_m to r_k, n_q the quadrature directions and w_q = 1 / N_quad.

Readings (the paper does not spell these out):
  E1  an electron interacts with the pseudopotential of a nucleus when it is
      within that nucleus's r_cut; r_cut is below half the smallest distance
      between pseudopotential nuclei, so at most one applies (the first in
      nucleus order if the caller breaks this).
  E2  quadrature rules: the vertices of the regular tetrahedron (N_quad = 4,
      exact to degree 2), octahedron (6, degree 3) and icosahedron (12,
      degree 5), equal weights, rotated by one random rotation per walker and
      electron.
  E3  the rotation: unit quaternion from three uniforms (Shoemake, "Uniform
      random rotations", Graphics Gems III, 1992),
      q = (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2, sqrt(u1) sin 2pi u3,
      sqrt(u1) cos 2pi u3) = (x, y, z, w); u1..u3 from words 0..2 of Philox
      counter (k, 0, walker, 3) under the 64-bit seed key of the sampler.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from . import fire_oracle as O
from .mcmc_oracle import MASK, philox4x32_10, u01

_G = (1.0 + math.sqrt(5.0)) / 2.0


def quadrature(n_quad: int):
    """(directions [Q, 3], weights [Q]) of reading E2 before rotation."""
    if n_quad == 4:
        d = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    elif n_quad == 6:
        d = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    elif n_quad == 12:
        d = []
        for a in (1.0, -1.0):
            for b in (_G, -_G):
                d += [[0.0, a, b], [a, b, 0.0], [b, 0.0, a]]
        d = np.array(d)
    else:
        raise ValueError(n_quad)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return d, np.full(n_quad, 1.0 / n_quad)


def rotation(seed: int, walker: int, k: int) -> np.ndarray:
    """3 x 3 rotation of reading E3."""
    key = (seed & MASK, (seed >> 32) & MASK)
    c = philox4x32_10((k, 0, walker, 3), key)
    u1, u2, u3 = (float(u01(c[t])) for t in range(3))
    x = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    y = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    z = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    w = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def legendre(l: int, x):
    if l == 0:
        return np.ones_like(x)
    if l == 1:
        return x
    if l == 2:
        return 1.5 * x * x - 0.5
    raise ValueError(l)


def v_channel(ecp: Dict, l: int, x) -> np.ndarray:
    """v_l(x) = sum_j c_j x^p_j exp(-a_j x^2) of one nucleus."""
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    for c, pw, a in ecp["terms"][l]:
        out = out + c * np.asarray(x, dtype=np.float64) ** pw * np.exp(-a * np.asarray(x) ** 2)
    return out


def nonlocal_energy(system, arch, params, r_np: np.ndarray, ecp: List[Dict], seed: int,
                    return_scale: bool = False):
    """V_nl per walker [W].  ecp[m] = None (no pseudopotential) or
    {"n_quad": 4|6|12, "r_cut": x, "terms": [[(c, p, a), ...] for l = 0..l_max]}.
    With return_scale, also the sum of the magnitudes of the summed terms
    (the scale a rounding error of the sum is relative to)."""
    r = np.asarray(r_np, dtype=np.float64)
    W, n = r.shape[0], r.shape[1]
    R = np.asarray(system.nuc_pos, dtype=np.float64)
    lp, sg = O.logpsi_np(system, arch, params, r)
    out = np.zeros(W)
    scale = np.zeros(W)
    for k in range(n):
        # the pseudopotential nucleus of electron k in every walker (E1)
        nuc = np.full(W, -1)
        for m in range(R.shape[0]):
            if ecp[m] is None:
                continue
            dist = np.linalg.norm(r[:, k] - R[m], axis=-1)
            nuc = np.where((nuc < 0) & (dist < ecp[m]["r_cut"]), m, nuc)
        for m in sorted(set(int(v) for v in nuc if v >= 0)):
            ws = np.nonzero(nuc == m)[0]
            e = ecp[m]
            base, wq = quadrature(e["n_quad"])
            rel = r[ws, k] - R[m]
            rad = np.linalg.norm(rel, axis=-1)
            rhat = rel / rad[:, None]
            dirs = np.stack([base @ rotation(seed, int(w), k).T for w in ws])     # [Wm, Q, 3]
            cos = np.einsum("wqx,wx->wq", dirs, rhat)
            ratio = np.zeros((ws.size, e["n_quad"]))
            for q in range(e["n_quad"]):
                rp = r[ws].copy()
                rp[:, k] = R[m] + rad[:, None] * dirs[:, q]
                lpn, sgn = O.logpsi_np(system, arch, params, rp)
                ratio[:, q] = sgn * sg[ws] * np.exp(lpn - lp[ws])
            for l in range(len(e["terms"])):
                term = v_channel(e, l, rad)[:, None] * (2 * l + 1) * wq * legendre(l, cos) * ratio
                out[ws] += term.sum(-1)
                scale[ws] += np.abs(term).sum(-1)
    return (out, scale) if return_scale else out
