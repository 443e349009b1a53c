"""Parameter recipes that reduce the ansatz to closed forms (shared by the
oracle pins and the GPU tests)."""
import numpy as np

from paper_2504_06087_gb300 import synth


def const_h_params(system, arch, seed=0, bias=1.0):
    """Parameters that make every embedding h_i the same constant vector.

    nuc_emb = 0 and the feature weights 0 make the filter sum vanish, so
    LN(0) = beta = 0 and h^0 = GLU(0) = 0; zero message weights keep h^1 = 0;
    zero MLP matrices with bias b give h = L * SiLU(b) in every component.
    """
    p = synth.init_params(system, arch, seed)
    p["nuc_emb"][:] = 0.0
    p["en_wfeat"][:] = 0.0
    p["msg_w"][:] = 0.0
    p["msg_b"][:] = 0.0
    p["mlp_w"][:] = 0.0
    p["mlp_b"][:] = bias
    return p


def hydrogen_like(sigma=1.0, z=1.0, width=8):
    """One electron on a charge-z nucleus with Psi = exp(-sigma r) exactly:
    constant embeddings, one determinant of one envelope orbital, no Jastrow.
    (The CUDA path takes widths that are multiples of 32.)"""
    system = synth.System(np.zeros((1, 3)), np.array([z]), 1, 1, 5.0, 20.0, "H")
    arch = synth.Arch(width=width, n_layers=1, n_det=1, n_env=1, jastrow_width=width, flags=0)
    p = const_h_params(system, arch)
    p["orb_w"][:] = 1.0
    p["env_pi"][:] = 1.0
    p["env_sigma"][:] = sigma
    return system, arch, p


def two_electron_product(z=2.0, s0=1.6, s1=0.9):
    """1 up + 1 down electron with Psi = c exp(-s0 |r_0|) exp(-s1 |r_1|): a
    diagonal 2 x 2 orbital matrix of two exponentials, no Jastrow."""
    system = synth.System(np.zeros((1, 3)), np.array([z]), 2, 1, 5.0, 20.0, "He")
    arch = synth.Arch(width=8, n_layers=2, n_det=1, n_env=2, jastrow_width=8, flags=0)
    p = const_h_params(system, arch)
    p["orb_w"][:] = 0.0
    p["orb_w"][0, 0, :, 0] = 1.0      # up-spin row uses orbital 0
    p["orb_w"][1, 0, :, 1] = 1.0      # down-spin row uses orbital 1
    p["env_pi"][:] = 0.0
    p["env_pi"][0, 0, 0, 0, :] = [1.0, 0.0]
    p["env_pi"][1, 0, 1, 0, :] = [0.0, 1.0]
    p["env_sigma"][0] = [s0, s1]
    return system, arch, p
