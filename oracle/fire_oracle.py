"""Plain FP64 CPU oracle of the FiRE wave function and its local energy.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path; both consume the seeded arrays of ``synth``.

Every quantity is computed from its definition in the paper, densely over all
electron pairs and all electron-nucleus pairs, and masked afterwards with the
cutoff polynomial and an explicit ``|x| <= c`` mask (Results, "Finite-range
embeddings": N_i = {j != i : |r_i - r_j| <= c}).  Gradients and Laplacians of
log|Psi| come from PyTorch autograd: the Laplacian is the trace of the exact
Hessian, one second-derivative pass per electron coordinate.  No step uses
the sparse forward Laplacian or low-rank updates the paper introduces; those
are what the CUDA path is checked against.

Readings where the paper is silent or garbled:
  R1  one message-passing round (Methods "Wave function ansatz"); "layers" is
      the depth L of the embedding MLP h = MLP(h^1).
  R2  GLU(x) = (SiLU(LN(x) W_g) * (LN(x) W_v)) W_o, LN over the width with
      learnable gamma, beta and eps = 1e-5, no biases.
  R3  the activation sigma is SiLU everywhere.
  R4  Gamma(x) = (SiLU(x W_1 + b_1) W_2) * (chi(x_0) W_env); W_1, b_1 per nucleus
      for the electron-nucleus filter; W_2, W_env, sigma_i shared.
  R5  f_cut(s) = 1 - (p+1)(p+2)/2 s^p + p(p+2) s^(p+1) - p(p+1)/2 s^(p+2),
      s = x / cutoff, p = 6, and 0 for s >= 1 (C^2 at the cutoff).
  R6  envelopes decay: phi_l(r) = sum_m sum_e pi_lme exp(-sigma_me |r - R_m|);
      sigma_me shared by all orbitals, determinants and spins.
  R7  full n x n determinants; rows of spin-up electrons use the up-spin
      orbital weights and envelope weights, rows of spin-down electrons the
      down-spin ones.
  R8  the Jastrow factors multiply: log|J| = cusp exponent
      + [sum_i MLP1(h_i) + log|sum_i MLP2(h_i)|] + [MLP1'(V) + log|MLP2'(V)|].
  R9  MLP(x) = w3 . SiLU(SiLU(x W1 + b1) W2 + b2) + b3 (two hidden layers).
  R10 attention scores h_i . q_r without scaling; softmax over electrons.
  R11 separate message weights W^alpha, b^alpha for parallel / antiparallel
      spins; the electron-electron filter Gamma is shared by both.
  R12 embedding MLP: L residual blocks h <- h + SiLU(h W_l + b_l).
  R13 the cutoff test is |r_i - r_j| <= c (equal values either way, since the
      filter vanishes at the cutoff).
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np
import torch

DT = torch.float64
LN_EPS = 1e-5
P_CUT = 6
J_CUSP, J_MLP, J_ATT = 1, 2, 4


def _t(x) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(DT)
    return torch.as_tensor(np.asarray(x), dtype=DT)


def params_to_torch(params: Dict[str, np.ndarray]) -> Dict[str, torch.Tensor]:
    return {k: _t(v) for k, v in params.items()}


# ---------------------------------------------------------------------------
# Building blocks
# ---------------------------------------------------------------------------

def silu(x: torch.Tensor) -> torch.Tensor:
    """sigma(x) = x * logistic(x) (reading R3)."""
    return x * torch.sigmoid(x)


def f_cut(s: torch.Tensor, p: int = P_CUT) -> torch.Tensor:
    """Polynomial cutoff of Gasteiger et al. (Methods, filter Gamma_m; R5)."""
    poly = (1.0 - (p + 1) * (p + 2) / 2.0 * s ** p + p * (p + 2) * s ** (p + 1)
            - p * (p + 1) / 2.0 * s ** (p + 2))
    return torch.where(s < 1.0, poly, torch.zeros_like(s))


def layer_norm(x: torch.Tensor, gamma: torch.Tensor, beta: torch.Tensor) -> torch.Tensor:
    """LayerNorm over the last axis (Ba et al.), biased variance, eps = 1e-5."""
    mu = x.mean(dim=-1, keepdim=True)
    var = ((x - mu) ** 2).mean(dim=-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + LN_EPS) * gamma + beta


def glu(x: torch.Tensor, p: Dict[str, torch.Tensor]) -> torch.Tensor:
    """Gated linear unit with LayerNorm (Methods, eq. of h^0_i; reading R2)."""
    y = layer_norm(x, p["ln_gamma"], p["ln_beta"])
    return (silu(y @ p["glu_wg"]) * (y @ p["glu_wv"])) @ p["glu_wo"]


def pair_features(delta: torch.Tensor, valid: torch.Tensor) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """e = Concat[|delta|, delta] and its rescaled form log(1+|e|)/|e| * e.

    ``valid`` marks pairs with delta != 0 by construction (i != j); the norm is
    evaluated through a double ``where`` so that the masked diagonal produces
    neither NaN values nor NaN derivatives.
    """
    d2 = (delta ** 2).sum(-1)
    safe = torch.where(valid, d2, torch.ones_like(d2))
    dist = torch.where(valid, torch.sqrt(safe), torch.zeros_like(d2))
    sdist = torch.sqrt(safe)
    e = torch.cat([dist[..., None], delta], dim=-1)
    scale = torch.where(valid, torch.log1p(sdist) / sdist, torch.zeros_like(d2))
    return e, scale[..., None] * e, dist


def radial_filter(e: torch.Tensor, w1: torch.Tensor, b1: torch.Tensor, w2: torch.Tensor,
                  wenv: torch.Tensor, sigma: torch.Tensor, cutoff: float) -> torch.Tensor:
    """Gamma(x) = SiLU(x W_1 + b_1) W_2 * chi(x_0) W_env (Methods; R4).

    chi(x) = f_cut(x / cutoff) * [exp(-sigma_i^2 x^2)]_i.  ``w1``/``b1`` may carry
    a leading per-nucleus axis aligned with ``e``'s second-to-last axis.
    """
    if w1.dim() == 3:      # per nucleus: e [..., N, 4], w1 [N, 4, H]
        u = torch.einsum("...mk,mkh->...mh", e, w1) + b1
    else:
        u = e @ w1 + b1
    g = silu(u) @ w2
    x0 = e[..., 0]
    if cutoff > 0:
        fc = f_cut(x0 / cutoff)
    else:
        fc = torch.zeros_like(x0)
    chi = fc[..., None] * torch.exp(-(sigma ** 2) * x0[..., None] ** 2)
    return g * (chi @ wenv)


def mlp_readout(x: torch.Tensor, p: Dict[str, torch.Tensor], pre: str) -> torch.Tensor:
    """Scalar MLP with two hidden layers (reading R9)."""
    a = silu(x @ p[pre + "_w1"] + p[pre + "_b1"])
    a = silu(a @ p[pre + "_w2"] + p[pre + "_b2"])
    return a @ p[pre + "_w3"] + p[pre + "_b3"][0]


# ---------------------------------------------------------------------------
# Embeddings (Methods, "Finite-range embeddings")
# ---------------------------------------------------------------------------

def spins(n_el: int, n_up: int) -> torch.Tensor:
    s = torch.zeros(n_el, dtype=torch.long)
    s[n_up:] = 1
    return s


def en_sum(system, p: Dict[str, torch.Tensor], r: torch.Tensor) -> torch.Tensor:
    """Argument of the GLU in h^0_i: sum_m Gamma_m(e^_im) * (h^nuc_m + e^bar_im W)
    (Methods, eq. of h^0_i), masked to |r_i - R_m| <= c_n.  [B, n, d]."""
    R = _t(system.nuc_pos)
    den = r[:, :, None, :] - R[None, None, :, :]                      # [B,n,N,3]
    valid_en = torch.ones(den.shape[:-1], dtype=torch.bool)
    e_en, eb_en, dist_en = pair_features(den, valid_en)
    gam = radial_filter(e_en, p["en_w1"], p["en_b1"], p["en_w2"], p["en_wenv"],
                        p["en_sigma"], system.cutoff_nuc)                  # [B,n,N,d]
    mask_en = (dist_en <= system.cutoff_nuc).to(DT)[..., None]
    feat = p["nuc_emb"][None, None] + eb_en @ p["en_wfeat"]
    return (mask_en * gam * feat).sum(dim=2)


def message_pass(system, p: Dict[str, torch.Tensor], r: torch.Tensor, h0: torch.Tensor) -> torch.Tensor:
    """h^1_i = h^0_i + m^par_i + m^anti_i, one round (Methods, eq. of m^alpha_i; R1, R11):
    m^alpha_i = sum_{j in N^alpha_i} Gamma(e_ij) * SiLU(Concat[h^0_i, h^0_j, e^bar_ij] W^alpha + b^alpha)."""
    B, n, _ = r.shape
    dee = r[:, :, None, :] - r[:, None, :, :]                           # r_i - r_j
    offdiag = ~torch.eye(n, dtype=torch.bool)[None].expand(B, n, n)
    e_ee, eb_ee, dist_ee = pair_features(dee, offdiag)
    gam_ee = radial_filter(e_ee, p["ee_w1"], p["ee_b1"], p["ee_w2"], p["ee_wenv"],
                           p["ee_sigma"], system.cutoff)                     # [B,n,n,d]
    within = offdiag & (dist_ee <= system.cutoff)
    sp = spins(n, system.n_up)
    same = (sp[:, None] == sp[None, :])[None].expand(B, n, n)
    cat = torch.cat([h0[:, :, None, :].expand(B, n, n, h0.shape[-1]),
                     h0[:, None, :, :].expand(B, n, n, h0.shape[-1]), eb_ee], dim=-1)
    h1 = h0
    for alpha, sel in ((0, same), (1, ~same)):
        z = cat @ p["msg_w"][alpha] + p["msg_b"][alpha]
        msg = gam_ee * silu(z)
        m = ((within & sel).to(DT)[..., None] * msg).sum(dim=2)
        h1 = h1 + m
    return h1


def embedding_mlp(arch, p: Dict[str, torch.Tensor], h1: torch.Tensor) -> torch.Tensor:
    """h = MLP(h^1): L residual blocks h <- h + SiLU(h W_l + b_l) (Methods; R12)."""
    h = h1
    for l in range(arch.n_layers):
        h = h + silu(h @ p["mlp_w"][l] + p["mlp_b"][l])
    return h


def embeddings(system, arch, p: Dict[str, torch.Tensor], r: torch.Tensor):
    """Return (h0, h1, h), each [B, n, d] (Methods, "Finite-range embeddings")."""
    h0 = glu(en_sum(system, p, r), p)
    h1 = message_pass(system, p, r, h0)
    return h0, h1, embedding_mlp(arch, p, h1)


# ---------------------------------------------------------------------------
# Orbitals, determinants, Jastrow factors
# ---------------------------------------------------------------------------

def orbitals(system, arch, p, r, h) -> torch.Tensor:
    """Phi_dil = (h_i W_dl) phi_dl(r_i)  ->  [B, D, n, n]  (Methods; R6, R7)."""
    R = _t(system.nuc_pos)
    sp = spins(system.n_el, system.n_up)
    dist = torch.sqrt(((r[:, :, None, :] - R[None, None]) ** 2).sum(-1))     # [B,n,N]
    q = torch.exp(-p["env_sigma"][None, None] * dist[..., None])            # [B,n,N,E]
    w = p["orb_w"][sp]                                                      # [n,D,d,n]
    pi = p["env_pi"][sp]                                                    # [n,D,n,N,E]
    o = torch.einsum("bik,idkl->bdil", h, w)
    env = torch.einsum("bime,idlme->bdil", q, pi)
    return o * env


def slater_part(system, arch, p, r, h):
    """Signed sum of determinants: (log|sum_d det Phi_d|, sign, per-det logs)."""
    phi = orbitals(system, arch, p, r, h)
    n = phi.shape[-1]
    if n > 128 and torch.backends.mkl.is_available():
        # one LAPACK factorisation per matrix: batched torch.linalg.slogdet
        # stalled on an x86 build whose LAPACK is MKL once several intra-op
        # threads ran (n = 180; n <= 128 ran); per matrix it does not, with
        # the same LU
        per = [torch.linalg.slogdet(m) for m in phi.reshape(-1, n, n)]
        sgn = torch.stack([x[0] for x in per]).reshape(phi.shape[:-2])     # [B,D]
        lad = torch.stack([x[1] for x in per]).reshape(phi.shape[:-2])
    else:
        sgn, lad = torch.linalg.slogdet(phi)                                # [B,D]
    lmax = lad.max(dim=1, keepdim=True).values.detach()
    lmax = torch.where(torch.isfinite(lmax), lmax, torch.zeros_like(lmax))
    ssum = (sgn * torch.exp(lad - lmax)).sum(dim=1)
    return lmax[:, 0] + torch.log(torch.abs(ssum)), torch.sign(ssum), (sgn, lad)


def cusp_jastrow(system, p, r) -> torch.Tensor:
    """Exponent of J_cusp: sum over pairs of w a^2 / (a + r_ij) (Methods)."""
    n, nu = system.n_el, system.n_up
    wpar, wanti, apar, aanti = p["cusp"][0], p["cusp"][1], p["cusp"][2], p["cusp"][3]
    out = torch.zeros(r.shape[0], dtype=DT)
    iu, ju = torch.triu_indices(n, n, offset=1)
    if iu.numel() == 0:
        return out
    rij = torch.sqrt(((r[:, iu] - r[:, ju]) ** 2).sum(-1))
    same = ((iu < nu) == (ju < nu)).to(DT)
    upar = wpar * apar ** 2 / (apar + rij)
    uanti = wanti * aanti ** 2 / (aanti + rij)
    return (same * upar + (1 - same) * uanti).sum(-1)


def mlp_jastrow(p, h) -> Tuple[torch.Tensor, torch.Tensor]:
    """log|J_MLP| and its sign: exp(sum_i MLP1(h_i)) * sum_i MLP2(h_i)."""
    f1 = mlp_readout(h, p, "jm1").sum(-1)
    f2 = mlp_readout(h, p, "jm2").sum(-1)
    return f1 + torch.log(torch.abs(f2)), torch.sign(f2)


def att_registers(arch, p, h) -> torch.Tensor:
    """V = Concat_r softmax(H q_r)^T H W^V_r  ->  [B, n_reg * d_reg] (R10)."""
    scores = torch.einsum("bik,rk->bri", h, p["att_q"])
    a = torch.softmax(scores, dim=-1)                                       # over electrons
    v = torch.einsum("bri,bik,rkc->brc", a, h, p["att_wv"])
    return v.reshape(h.shape[0], -1)


def att_jastrow(arch, p, h) -> Tuple[torch.Tensor, torch.Tensor]:
    V = att_registers(arch, p, h)
    g1 = mlp_readout(V, p, "ja1")
    g2 = mlp_readout(V, p, "ja2")
    return g1 + torch.log(torch.abs(g2)), torch.sign(g2)


def logpsi(system, arch, p, r) -> Tuple[torch.Tensor, torch.Tensor]:
    """(log|Psi|, sign Psi) for positions r [B, n, 3] (Methods eq. wf; R8)."""
    _, _, h = embeddings(system, arch, p, r)
    la, sg, _ = slater_part(system, arch, p, r, h)
    if arch.flags & J_CUSP:
        la = la + cusp_jastrow(system, p, r)
    if arch.flags & J_MLP:
        lj, sj = mlp_jastrow(p, h)
        la, sg = la + lj, sg * sj
    if arch.flags & J_ATT:
        lj, sj = att_jastrow(arch, p, h)
        la, sg = la + lj, sg * sj
    return la, sg


# ---------------------------------------------------------------------------
# Hamiltonian (Methods eq. hamiltonian) and local energy
# ---------------------------------------------------------------------------

def potential(system, r: torch.Tensor) -> torch.Tensor:
    """V = sum_{i<j} 1/r_ij - sum_{i,m} Z_m/|r_i-R_m| + sum_{m<n} Z_m Z_n/R_mn."""
    R, Z = _t(system.nuc_pos), _t(system.nuc_charge)
    n, N = system.n_el, system.n_nuc
    v = torch.zeros(r.shape[0], dtype=DT)
    for i in range(n):
        for j in range(i + 1, n):
            v = v + 1.0 / torch.sqrt(((r[:, i] - r[:, j]) ** 2).sum(-1))
        for m in range(N):
            v = v - Z[m] / torch.sqrt(((r[:, i] - R[m]) ** 2).sum(-1))
    for m in range(N):
        for k in range(m + 1, N):
            v = v + Z[m] * Z[k] / torch.sqrt(((R[m] - R[k]) ** 2).sum())
    return v


def local_energy(system, arch, params, r_np, return_parts: bool = False):
    """E_L = -1/2 (Laplacian log|Psi| + |grad log|Psi||^2) + V (Methods).

    Returns numpy arrays (e_loc, logabs, sign[, e_kin, e_pot, grad, lap]).
    The Laplacian is the exact trace of the Hessian of log|Psi| with respect
    to all 3 n electron coordinates, one autograd pass per coordinate.
    """
    p = params_to_torch(params) if not isinstance(next(iter(params.values())), torch.Tensor) else params
    r = _t(r_np).clone().requires_grad_(True)
    la, sg = logpsi(system, arch, p, r)
    (g,) = torch.autograd.grad(la.sum(), r, create_graph=True)
    lap = torch.zeros(r.shape[0], dtype=DT)
    n = r.shape[1]
    for i in range(n):
        for x in range(3):
            (gg,) = torch.autograd.grad(g[:, i, x].sum(), r, retain_graph=True)
            lap = lap + gg[:, i, x].detach()
    g = g.detach()
    with torch.no_grad():
        v = potential(system, r.detach())
        kin = -0.5 * (lap + (g ** 2).sum(dim=(1, 2)))
        e = kin + v
    out = (e.numpy(), la.detach().numpy(), sg.detach().numpy())
    if return_parts:
        out = out + (kin.numpy(), v.numpy(), g.numpy(), lap.numpy())
    return out


def logpsi_np(system, arch, params, r_np):
    p = params_to_torch(params)
    with torch.no_grad():
        la, sg = logpsi(system, arch, p, _t(r_np))
    return la.numpy(), sg.numpy()


def grad_logpsi(system, arch, params, r_np, names=None):
    """Per-walker d log|Psi| / d theta, as a dict name -> [B, *shape] (Methods eq. spring)."""
    names = list(params.keys()) if names is None else names
    out = {k: [] for k in names}
    r = _t(r_np)
    for b in range(r.shape[0]):
        p = {k: _t(v).clone().requires_grad_(k in names) for k, v in params.items()}
        la, _ = logpsi(system, arch, p, r[b:b + 1])
        gs = torch.autograd.grad(la.sum(), [p[k] for k in names], allow_unused=True)
        for k, gk in zip(names, gs):
            out[k].append(torch.zeros_like(p[k]) if gk is None else gk.detach())
    return {k: torch.stack(v).numpy() for k, v in out.items()}
