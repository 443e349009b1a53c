"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds only input generation: molecule geometries, walker
positions and the initial parameter set of the FiRE ansatz (its names, shapes
and initial distributions).  It holds none of the method's arithmetic; both
the oracle and the CUDA path consume its arrays without importing each other.

Workloads (the paper times cumulenes on one A100 with 4096 walkers, Methods
"Measuring speedups"; these seeded molecules stand in for them):

* water: O (Z=8) at the origin, H (Z=1) at (1.81, 0, 0) and (-0.45, 1.75, 0)
  bohr, 10 electrons (5 up, 5 down).
* zigzag polyenes C_k H_(k+2): carbon j at (j*2.6*cos30, (j mod 2)*2.6*sin30, 0)
  (C-C 2.6 bohr at 120 degrees); every interior carbon carries one H at
  2.05 bohr along -y (even j) or +y (odd j); each terminal carbon carries two H
  at +-120 degrees from its C-C bond.  ``terminal_h=False`` drops the terminal
  hydrogens (C26H24: 180 electrons, 90 up / 90 down).
* walkers: every electron picks a nucleus with probability proportional to Z
  and adds an isotropic N(0, 1 bohr^2) displacement; the first n_up electrons
  are spin-up (Methods, "Variational Monte Carlo").
"""
from __future__ import annotations

import dataclasses
import math
import re
from typing import Dict, List, Tuple

import numpy as np

# Jastrow switches (Methods, "Global electron correlation effects").
J_CUSP = 1
J_MLP = 2
J_ATT = 4
J_ALL = J_CUSP | J_MLP | J_ATT


@dataclasses.dataclass
class System:
    """Nuclei, electron counts and cutoffs of one molecule."""

    nuc_pos: np.ndarray          # [N, 3] float64, bohr
    nuc_charge: np.ndarray       # [N] float64
    n_el: int
    n_up: int
    cutoff: float = 5.0          # c, electron-electron cutoff (bohr)
    cutoff_nuc: float = 20.0     # c_n, electron-nucleus cutoff (bohr)
    name: str = ""

    @property
    def n_nuc(self) -> int:
        return int(self.nuc_pos.shape[0])


@dataclasses.dataclass
class Arch:
    """Network hyper-parameters (Supplementary "Hyperparameters" table)."""

    width: int = 256             # hidden width d
    n_layers: int = 4            # depth L of the embedding MLP h = MLP(h^1)
    n_det: int = 4               # N_det
    n_env: int = 8               # envelopes per nucleus
    n_gauss: int = 32            # d_0, Gaussians of the radial filter
    edge_hidden: int = 16        # hidden width of the filter MLP
    jastrow_width: int = 0       # hidden width of the Jastrow MLPs (0 -> width)
    n_reg: int = 16              # attention registers
    d_reg: int = 16              # register dimension
    flags: int = J_ALL

    @property
    def jw(self) -> int:
        return self.jastrow_width if self.jastrow_width > 0 else self.width


# --------------------------------------------------------------------------
# Molecules
# --------------------------------------------------------------------------

def water(cutoff: float = 5.0, cutoff_nuc: float = 20.0) -> System:
    pos = np.array([[0.0, 0.0, 0.0], [1.81, 0.0, 0.0], [-0.45, 1.75, 0.0]])
    z = np.array([8.0, 1.0, 1.0])
    return System(pos, z, 10, 5, cutoff, cutoff_nuc, "water")


def zigzag_polyene(k: int, terminal_h: bool = True, cutoff: float = 5.0,
                   cutoff_nuc: float = 20.0) -> System:
    cc, ch = 2.6, 2.05
    # exact forms (sqrt is correctly rounded on every platform, unlike cos/sin)
    c30, s30 = math.sqrt(3.0) / 2.0, 0.5
    carbons = [np.array([j * cc * c30, (j % 2) * cc * s30, 0.0]) for j in range(k)]
    hyd: List[np.ndarray] = []
    for j in range(k):
        terminal = (j == 0 or j == k - 1)
        if terminal and k > 1:
            if not terminal_h:
                continue
            other = carbons[1] if j == 0 else carbons[k - 2]
            b = other - carbons[j]
            b = b / np.linalg.norm(b)
            for sn in (1.0, -1.0):      # rotations by +-120 degrees
                ca, sa = -0.5, sn * math.sqrt(3.0) / 2.0
                rb = np.array([ca * b[0] - sa * b[1], sa * b[0] + ca * b[1], 0.0])
                hyd.append(carbons[j] + ch * rb)
        else:
            sgn = -1.0 if j % 2 == 0 else 1.0
            hyd.append(carbons[j] + np.array([0.0, sgn * ch, 0.0]))
    pos = np.array(carbons + hyd)
    z = np.array([6.0] * k + [1.0] * len(hyd))
    n_el = int(round(z.sum()))
    name = f"C{k}H{len(hyd)}"
    return System(pos, z, n_el, (n_el + 1) // 2, cutoff, cutoff_nuc, name)


def hydrogen_atom() -> System:
    return System(np.zeros((1, 3)), np.array([1.0]), 1, 1, 5.0, 20.0, "H")


# --------------------------------------------------------------------------
# Walkers
# --------------------------------------------------------------------------

def walkers(system: System, n_walkers: int, seed: int) -> np.ndarray:
    """[W, n_el, 3] float64 electron positions (nucleus chosen with p ~ Z)."""
    rng = np.random.default_rng(seed)
    p = system.nuc_charge / system.nuc_charge.sum()
    nuc = rng.choice(system.n_nuc, size=(n_walkers, system.n_el), p=p)
    r = system.nuc_pos[nuc] + rng.standard_normal((n_walkers, system.n_el, 3))
    return np.ascontiguousarray(r, dtype=np.float64)


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------

def param_spec(system: System, arch: Arch) -> List[Tuple[str, Tuple[int, ...]]]:
    """Ordered (name, shape) list of every trainable array of the ansatz."""
    n, N = system.n_el, system.n_nuc
    d, L, D, E = arch.width, arch.n_layers, arch.n_det, arch.n_env
    G, H, J = arch.n_gauss, arch.edge_hidden, arch.jw
    R, dr = arch.n_reg, arch.d_reg
    spec: List[Tuple[str, Tuple[int, ...]]] = [
        # electron-nucleus filter Gamma_m and initial embedding h^0
        ("en_w1", (N, 4, H)), ("en_b1", (N, H)), ("en_w2", (H, d)),
        ("en_wenv", (G, d)), ("en_sigma", (G,)),
        ("nuc_emb", (N, d)), ("en_wfeat", (4, d)),
        ("ln_gamma", (d,)), ("ln_beta", (d,)),
        ("glu_wg", (d, d)), ("glu_wv", (d, d)), ("glu_wo", (d, d)),
        # electron-electron filter Gamma and the message passing step
        ("ee_w1", (4, H)), ("ee_b1", (H,)), ("ee_w2", (H, d)),
        ("ee_wenv", (G, d)), ("ee_sigma", (G,)),
        ("msg_w", (2, 2 * d + 4, d)), ("msg_b", (2, d)),
        # embedding MLP
        ("mlp_w", (L, d, d)), ("mlp_b", (L, d)),
        # orbitals and envelopes (spin, determinant)
        ("orb_w", (2, D, d, n)), ("env_pi", (2, D, n, N, E)), ("env_sigma", (N, E)),
        # Jastrow factors
        ("cusp", (4,)),
    ]
    for pre, din in (("jm1", d), ("jm2", d), ("ja1", R * dr), ("ja2", R * dr)):
        spec += [(pre + "_w1", (din, J)), (pre + "_b1", (J,)),
                 (pre + "_w2", (J, J)), (pre + "_b2", (J,)),
                 (pre + "_w3", (J,)), (pre + "_b3", (1,))]
        if pre == "jm2":
            spec += [("att_q", (R, d)), ("att_wv", (R, d, dr))]
    return spec


def _geometric_inv(g: int, lo: float, hi: float) -> np.ndarray:
    s = lo * (hi / lo) ** (np.arange(g) / max(g - 1, 1))
    return 1.0 / s


def init_params(system: System, arch: Arch, seed: int) -> Dict[str, np.ndarray]:
    """Seeded initial parameters: every matrix N(0, 1/fan_in), biases 0.

    Special initialisations: Gaussian widths 1/s with s geometric from 0.5 to
    the filter cutoff; envelope exponents Z_m (e+1)/N_env; envelope weights
    N(0, 1/(N_nuc N_env)); nuclear embeddings N(0, 1); LayerNorm gamma=1,
    beta=0; cusp Jastrow (w_par, w_anti, a_par, a_anti) = (-1/4, -1/2, 1, 1).
    """
    rng = np.random.default_rng(seed)
    out: Dict[str, np.ndarray] = {}
    for name, shape in param_spec(system, arch):
        if name in ("en_sigma",):
            v = _geometric_inv(shape[0], 0.5, system.cutoff_nuc)
        elif name in ("ee_sigma",):
            v = _geometric_inv(shape[0], 0.5, max(system.cutoff, 0.5))
        elif name == "env_sigma":
            e = np.arange(shape[1]) + 1.0
            v = system.nuc_charge[:, None] * e[None, :] / shape[1]
        elif name == "env_pi":
            v = rng.standard_normal(shape) / math.sqrt(shape[3] * shape[4])
        elif name == "nuc_emb":
            v = rng.standard_normal(shape)
        elif name == "ln_gamma":
            v = np.ones(shape)
        elif name == "ln_beta":
            v = np.zeros(shape)
        elif name == "cusp":
            v = np.array([-0.25, -0.5, 1.0, 1.0])
        elif re.search(r"_b\d?$", name):
            v = np.zeros(shape)
        elif name == "en_w1":
            v = rng.standard_normal(shape) / math.sqrt(shape[1])
        elif name in ("msg_w", "orb_w", "mlp_w", "att_wv"):
            v = rng.standard_normal(shape) / math.sqrt(shape[-2])
        elif name == "att_q":
            v = rng.standard_normal(shape) / math.sqrt(shape[-1])
        elif name.endswith("_w3"):
            v = rng.standard_normal(shape) / math.sqrt(shape[0])
        else:  # plain [fan_in, fan_out] matrices
            v = rng.standard_normal(shape) / math.sqrt(shape[0])
        out[name] = np.ascontiguousarray(v, dtype=np.float64)
    return out


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    key: str
    index: int            # seed base: walkers use 1000+index, parameters index
    system: System
    arch: Arch
    n_walkers: int
    precision: str        # "fp64", "fp32" or "bf16"


def workload(key: str, n_walkers: int | None = None) -> Workload:
    if key == "water":
        w = Workload(key, 1, water(), Arch(width=64, n_layers=2, n_det=4), 256, "fp64")
    elif key == "c8h10":
        w = Workload(key, 2, zigzag_polyene(8), Arch(width=128, n_layers=3, n_det=8), 4096, "fp32")
    elif key == "c26h24":
        w = Workload(key, 3, zigzag_polyene(26, terminal_h=False),
                     Arch(width=256, n_layers=4, n_det=16), 4096, "bf16")
    elif key.startswith("sample_k"):
        k = int(key[len("sample_k"):])
        w = Workload(key, 5, zigzag_polyene(k), Arch(width=256, n_layers=4, n_det=16), 4096, "fp32")
    else:
        raise KeyError(key)
    if n_walkers is not None:
        w.n_walkers = n_walkers
    return w


def make_inputs(w: Workload, n_walkers: int | None = None):
    """(positions [W,n,3], parameter dict) for a workload, fully seeded."""
    nw = w.n_walkers if n_walkers is None else n_walkers
    r = walkers(w.system, nw, 1000 + w.index)
    p = init_params(w.system, w.arch, w.index)
    return r, p
