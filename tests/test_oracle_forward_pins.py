"""Hand-worked pins of the oracle's forward formulas (Methods, "Wave function
ansatz": the equations of h^0_i, Gamma_m, chi, m^alpha_i, h = MLP(h^1),
J_MLP and J_att).

Every case is tiny (width 2, one to three electrons) with weights chosen so
that each term of the formula is non-zero and the activations land on points
where SiLU has a closed form: SiLU(ln a) = ln a * a / (1 + a), so
SiLU(ln 3) = 3/4 ln 3, SiLU(-ln 3) = -1/4 ln 3, SiLU(ln 7) = 7/8 ln 7.  The
expected values are written out as scalars from those closed forms; none of
them calls the oracle.  tests/test_oracle_mutations.py plants plausible
mistakes (swapped operands, a dropped square, a reordered concatenation, a
missing rescale or residual) in the oracle and checks that these pins fail.
"""
import math

import numpy as np
import pytest
import torch

from paper_2504_06087_gb300 import synth
from oracle import fire_oracle as O

L3, L7, L2 = math.log(3.0), math.log(7.0), math.log(2.0)
EPS = 1e-5
TOL = 1e-13


def T(x):
    return torch.tensor(x, dtype=torch.float64)


def silu_closed(x):
    """Scalar SiLU x / (1 + e^-x) for points without a nicer form."""
    return x / (1.0 + math.exp(-x))


# f_cut at s = 1/2 and s = 1/4 (p = 6), fractions worked by hand:
# 1 - 28 s^6 + 48 s^7 - 21 s^8
FC_HALF = (256 - 112 + 96 - 21) / 256.0            # = 219/256
FC_QUARTER = (65536 - 448 + 192 - 21) / 65536.0    # = 65259/65536


def test_fcut_hand_values():
    """Reading R5 at two interior points (the fractions above)."""
    got = O.f_cut(T([0.5, 0.25]))
    assert abs(float(got[0]) - FC_HALF) < TOL and abs(float(got[1]) - FC_QUARTER) < TOL


# ---------------------------------------------------------------------------
# GLU with LayerNorm (reading R2)
# ---------------------------------------------------------------------------

def glu_case():
    s = 1.0 / math.sqrt(1.0 + EPS)          # LN([1, -1]) = [s, -s]: mean 0, variance 1
    p = {"ln_gamma": T([1.0, 1.0]), "ln_beta": T([0.0, 0.0]),
         "glu_wg": T([[L3 / s, 0.0], [0.0, 0.0]]),        # LN(x) W_g = [ln 3, 0]
         "glu_wv": T([[2.0 / s, 0.0], [0.0, 5.0 / s]]),   # LN(x) W_v = [2, -5]
         "glu_wo": T([[1.0, -2.0], [3.0, 4.0]])}
    return T([[1.0, -1.0]]), p


def test_glu_hand_case():
    """(SiLU(LN(x) W_g) * LN(x) W_v) W_o = ([3/4 ln 3, 0] * [2, -5]) W_o
    = [3/2 ln 3, 0] W_o = [3/2 ln 3, -3 ln 3]."""
    x, p = glu_case()
    got = O.glu(x, p)[0]
    want = [1.5 * L3, -3.0 * L3]
    assert abs(float(got[0]) - want[0]) < TOL and abs(float(got[1]) - want[1]) < TOL


def test_glu_layer_norm_uses_gamma_and_beta():
    """gamma = [2, 1], beta = [ln 3 - 2s, 0]: LN(x) = [ln 3, -s], so with
    W_g = W_v = I the gate gives [3/4 ln 3 * ln 3, SiLU(-s) * (-s)]."""
    s = 1.0 / math.sqrt(1.0 + EPS)
    p = {"ln_gamma": T([2.0, 1.0]), "ln_beta": T([L3 - 2 * s, 0.0]),
         "glu_wg": T(np.eye(2)), "glu_wv": T(np.eye(2)), "glu_wo": T(np.eye(2))}
    got = O.glu(T([[1.0, -1.0]]), p)[0]
    want = [0.75 * L3 * L3, silu_closed(-s) * (-s)]
    assert abs(float(got[0]) - want[0]) < TOL and abs(float(got[1]) - want[1]) < TOL


# ---------------------------------------------------------------------------
# pair features and their rescale (Methods, e_ij, e^_im and e^bar)
# ---------------------------------------------------------------------------

def test_pair_features_hand_case():
    """delta = (0, 3, 4): e = [5, 0, 3, 4], e^bar = ln(6)/5 * e = ln 6 [1, 0, 3/5, 4/5];
    delta = (-2, 0, 0): e^bar = ln(3)/2 * [2, -2, 0, 0]; masked pairs give zeros."""
    delta = T([[0.0, 3.0, 4.0], [-2.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    valid = torch.tensor([True, True, False])
    e, eb, dist = O.pair_features(delta, valid)
    L6 = math.log(6.0)
    np.testing.assert_allclose(e[0].numpy(), [5, 0, 3, 4], atol=TOL)
    np.testing.assert_allclose(eb[0].numpy(), [L6, 0, 0.6 * L6, 0.8 * L6], atol=TOL)
    np.testing.assert_allclose(eb[1].numpy(), [L3, -L3, 0, 0], atol=TOL)
    np.testing.assert_allclose(dist.numpy(), [5, 2, 0], atol=TOL)
    assert torch.all(eb[2] == 0) and torch.all(e[2] == 0)


# ---------------------------------------------------------------------------
# radial filter Gamma (Methods, Gamma_m and chi; readings R4, R5)
# ---------------------------------------------------------------------------

def filter_params():
    """Nucleus 0: x W_1 + b_1 = [ln 3, -ln 3] for x = [1, 0.6, 0.8, 0];
    nucleus 1: W_1 = 0, b_1 = [ln 7, 0].  W_2 = [[1, 1], [2, 4]],
    W_env = [[1, 1], [0, 2]], sigma = [1, 1/2] (d_0 = 2, hidden width 2)."""
    w1 = np.zeros((2, 4, 2))
    w1[0, 0, 0] = L3
    w1[0, 1, 1] = 5.0 / 3.0 * L3
    b1 = np.array([[0.0, -2.0 * L3], [L7, 0.0]])
    return (T(w1), T(b1), T([[1.0, 1.0], [2.0, 4.0]]), T([[1.0, 1.0], [0.0, 2.0]]), T([1.0, 0.5]))


def gamma_closed(nucleus, x0, fc):
    """Gamma for the filter_params() of one nucleus at distance x0, written out:
    SiLU(u) W_2 with u = [ln 3, -ln 3] (nucleus 0) or [ln 7, 0] (nucleus 1), and
    chi W_env = fc [e^{-x0^2}, e^{-x0^2} + 2 e^{-x0^2/4}]."""
    if nucleus == 0:
        a = [0.75 * L3, -0.25 * L3]
    else:
        a = [0.875 * L7, 0.0]
    g = [a[0] * 1 + a[1] * 2, a[0] * 1 + a[1] * 4]
    c0, c1 = math.exp(-x0 ** 2), math.exp(-(0.5 * x0) ** 2)
    env = [fc * c0, fc * (c0 + 2 * c1)]
    return [g[0] * env[0], g[1] * env[1]]


def test_radial_filter_hand_case():
    w1, b1, w2, wenv, sig = filter_params()
    e = T([[1.0, 0.6, 0.8, 0.0]])
    got = O.radial_filter(e, w1[0], b1[0], w2, wenv, sig, 2.0)[0]     # x0 / c = 1/2
    want = gamma_closed(0, 1.0, FC_HALF)
    np.testing.assert_allclose(got.numpy(), want, rtol=0, atol=TOL)


def test_radial_filter_per_nucleus_weights():
    """Per-nucleus W_1, b_1 (the electron-nucleus filter Gamma_m): each nucleus
    applies its own first layer; beyond the cutoff the filter is zero."""
    w1, b1, w2, wenv, sig = filter_params()
    e = T([[[1.0, 0.6, 0.8, 0.0], [2.0, 0.0, 0.0, 2.0]],
           [[1.0, 0.6, 0.8, 0.0], [4.5, 0.0, 0.0, 4.5]]])
    got = O.radial_filter(e, w1, b1, w2, wenv, sig, 4.0)
    np.testing.assert_allclose(got[0, 0].numpy(), gamma_closed(0, 1.0, FC_QUARTER), atol=TOL)
    np.testing.assert_allclose(got[0, 1].numpy(), gamma_closed(1, 2.0, FC_HALF), atol=TOL)
    assert torch.all(got[1, 1] == 0.0)


# ---------------------------------------------------------------------------
# initial embedding: the sum over nuclei before the GLU (Methods, h^0_i)
# ---------------------------------------------------------------------------

def test_electron_nucleus_sum_hand_case():
    """One electron at (0.6, 0.8, 0); nucleus 0 at the origin (distance 1),
    nucleus 1 at (0.6, 0.8, -2) (distance 2), c_n = 4.  e^bar W_feat with
    W_feat picking components 0 and 3: [ln 2, 0] and [ln 3, ln 3];
    nuclear embeddings [2, 3] and [-1, 5]."""
    w1, b1, w2, wenv, sig = filter_params()
    system = synth.System(np.array([[0.0, 0.0, 0.0], [0.6, 0.8, -2.0]]), np.array([1.0, 1.0]),
                          1, 1, 5.0, 4.0, "x")
    wf = np.zeros((4, 2))
    wf[0, 0] = 1.0
    wf[3, 1] = 1.0
    p = {"en_w1": w1, "en_b1": b1, "en_w2": w2, "en_wenv": wenv, "en_sigma": sig,
         "nuc_emb": T([[2.0, 3.0], [-1.0, 5.0]]), "en_wfeat": T(wf)}
    r = T([[[0.6, 0.8, 0.0]]])
    got = O.en_sum(system, p, r)[0, 0]
    g0 = gamma_closed(0, 1.0, FC_QUARTER)
    g1 = gamma_closed(1, 2.0, FC_HALF)
    feat0 = [2.0 + L2, 3.0]
    feat1 = [-1.0 + L3, 5.0 + L3]
    want = [g0[0] * feat0[0] + g1[0] * feat1[0], g0[1] * feat0[1] + g1[1] * feat1[1]]
    np.testing.assert_allclose(got.numpy(), want, rtol=0, atol=TOL)


# ---------------------------------------------------------------------------
# message passing (Methods, m^alpha_i; readings R1, R11, R13)
# ---------------------------------------------------------------------------

def message_params(active):
    """Gamma(e_ij) = [3/4 ln 3 fc e^-1, -1/4 ln 3 fc e^-1/4] at |r_ij| = 2
    (W_1 = 0, b_1 = [ln 3, -ln 3], W_2 = W_env = I, sigma = [1/2, 1/4]).
    The active channel's W maps Concat[h0_i, h0_j, e^bar_ij] to
    z = [ln 7 h0_i[0], ln 7 h0_j[1] + e^bar_ij[1]]; the idle channel's weights
    are ones with bias 5 (any use of them changes the result)."""
    w = np.ones((2, 8, 2))
    b = np.full((2, 2), 5.0)
    w[active] = 0.0
    b[active] = 0.0
    w[active, 0, 0] = L7       # h0_i[0] -> z[0]
    w[active, 3, 1] = L7       # h0_j[1] -> z[1]
    w[active, 5, 1] = 1.0      # e^bar_ij[1] -> z[1]
    return {"ee_w1": T(np.zeros((4, 2))), "ee_b1": T([L3, -L3]), "ee_w2": T(np.eye(2)),
            "ee_wenv": T(np.eye(2)), "ee_sigma": T([0.5, 0.25]), "msg_w": T(w), "msg_b": T(b)}


def message_expected():
    """Electrons 0 at the origin and 1 at (2, 0, 0) (c = 4, f_cut = 219/256),
    h0_0 = [1, 0], h0_1 = [0, 1]; e^bar_01 = ln 3 [1, -1, 0, 0],
    e^bar_10 = ln 3 [1, 1, 0, 0].
    z_01 = [ln 7, ln 7 - ln 3] -> SiLU = [7/8 ln 7, 7/10 ln(7/3)];
    z_10 = [0, ln 3] -> SiLU = [0, 3/4 ln 3]."""
    gam = [0.75 * L3 * FC_HALF * math.exp(-1.0), -0.25 * L3 * FC_HALF * math.exp(-0.25)]
    m0 = [gam[0] * 0.875 * L7, gam[1] * 0.7 * math.log(7.0 / 3.0)]
    m1 = [0.0, gam[1] * 0.75 * L3]
    return [1.0 + m0[0], m0[1]], [m1[0], 1.0 + m1[1]]


@pytest.mark.parametrize("n_up,active", [(3, 0), (1, 1)])
def test_message_pass_hand_case(n_up, active):
    """Same-spin pairs use W^par (channel 0), opposite-spin pairs W^anti
    (channel 1).  A third electron 10 bohr away, beyond c, receives and sends
    nothing (with n_up = 1 it shares the spin of electron 1)."""
    system = synth.System(np.zeros((1, 3)), np.array([1.0]), 3, n_up, 4.0, 20.0, "x")
    p = message_params(active)
    r = T([[[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [10.0, 0.0, 0.0]]])
    h0 = T([[[1.0, 0.0], [0.0, 1.0], [3.0, -1.0]]])
    got = O.message_pass(system, p, r, h0)[0]
    h10, h11 = message_expected()
    np.testing.assert_allclose(got[0].numpy(), h10, rtol=0, atol=TOL)
    np.testing.assert_allclose(got[1].numpy(), h11, rtol=0, atol=TOL)
    np.testing.assert_allclose(got[2].numpy(), [3.0, -1.0], rtol=0, atol=0)


# ---------------------------------------------------------------------------
# embedding MLP (reading R12) and the scalar readout MLP (reading R9)
# ---------------------------------------------------------------------------

def test_embedding_mlp_hand_case():
    """h1 = [ln 3, 0]; block 1 (W = I, b = 0): h = [ln 3 + 3/4 ln 3, 0];
    block 2 maps h to [0, ln 7]: h = [7/4 ln 3, 7/8 ln 7]."""
    arch = synth.Arch(width=2, n_layers=2)
    w = np.zeros((2, 2, 2))
    w[0] = np.eye(2)
    w[1, 0, 1] = L7 / (1.75 * L3)
    p = {"mlp_w": T(w), "mlp_b": T(np.zeros((2, 2)))}
    got = O.embedding_mlp(arch, p, T([[ [L3, 0.0] ]]))[0, 0]
    np.testing.assert_allclose(got.numpy(), [1.75 * L3, 0.875 * L7], rtol=0, atol=TOL)


def readout_params(pre):
    """MLP(x) = w3 . SiLU(SiLU(x W1 + b1) W2 + b2) + b3 with W1 = I,
    b1 = [0, ln 7], W2 = [[1, 0], [0, 0]], b2 = [1/4 ln 3, -ln 3],
    w3 = [2, 4], b3 = 1/2."""
    return {pre + "_w1": T(np.eye(2)), pre + "_b1": T([0.0, L7]),
            pre + "_w2": T([[1.0, 0.0], [0.0, 0.0]]), pre + "_b2": T([0.25 * L3, -L3]),
            pre + "_w3": T([2.0, 4.0]), pre + "_b3": T([0.5])}


def readout_closed(x0):
    """The readout_params() MLP at x = [x0, anything]: layer 1 = [SiLU(x0), 7/8 ln 7],
    layer 2 = [SiLU(SiLU(x0) + 1/4 ln 3), -1/4 ln 3]."""
    a = silu_closed(x0)
    return 2.0 * silu_closed(a + 0.25 * L3) + 4.0 * (-0.25 * L3) + 0.5


def test_mlp_readout_hand_case():
    """At x = [ln 3, 0]: layer 1 = [3/4 ln 3, 7/8 ln 7], layer 2 = SiLU([ln 3, -ln 3])
    = [3/4 ln 3, -1/4 ln 3], output 3/2 ln 3 - ln 3 + 1/2."""
    p = readout_params("jm1")
    got = O.mlp_readout(T([[L3, 0.0]]), p, "jm1")
    assert abs(float(got[0]) - (0.5 * L3 + 0.5)) < TOL
    assert abs(readout_closed(L3) - (0.5 * L3 + 0.5)) < TOL


# ---------------------------------------------------------------------------
# Jastrow factors (Methods, J_MLP and J_att; readings R8-R10)
# ---------------------------------------------------------------------------

def jm2_params():
    """MLP_2 = 3/4 ln 3 - 1 < 0 for every input (W1 = W2 = 0, b2 = [ln 3, 0],
    w3 = [1, 0], b3 = -1)."""
    return {"jm2_w1": T(np.zeros((2, 2))), "jm2_b1": T([0.0, 0.0]),
            "jm2_w2": T(np.zeros((2, 2))), "jm2_b2": T([L3, 0.0]),
            "jm2_w3": T([1.0, 0.0]), "jm2_b3": T([-1.0])}


def test_mlp_jastrow_hand_case():
    """J_MLP = exp(sum_i MLP_1(h_i)) * sum_i MLP_2(h_i) with two electrons:
    log|J| = MLP_1(h_0) + MLP_1(h_1) + ln|2 (3/4 ln 3 - 1)|, sign -1."""
    p = dict(readout_params("jm1"), **jm2_params())
    h = T([[[L3, 0.0], [0.0, 0.0]]])
    lj, sj = O.mlp_jastrow(p, h)
    want = (0.5 * L3 + 0.5) + readout_closed(0.0) + math.log(abs(2.0 * (0.75 * L3 - 1.0)))
    assert abs(float(lj[0]) - want) < TOL
    assert float(sj[0]) == -1.0


def att_params():
    """Two registers, d_reg = 2: q_1 = [1, 0], q_2 = [0, 1]; W^V_1 = I,
    W^V_2 swaps the two components."""
    return {"att_q": T([[1.0, 0.0], [0.0, 1.0]]),
            "att_wv": T(np.array([np.eye(2), [[0.0, 1.0], [1.0, 0.0]]]))}


def test_attention_registers_hand_case():
    """h_0 = [ln 3, 0], h_1 = [0, 0]: scores of register 1 are [ln 3, 0], so the
    softmax over electrons is [3/4, 1/4] and v_1 = [3/4 ln 3, 0]; register 2
    scores [0, 0] (uniform) and v_2 = 1/2 (h_0 + h_1) W^V_2 = [0, 1/2 ln 3].
    V = Concat[v_1, v_2]."""
    arch = synth.Arch(width=2, n_layers=1, n_reg=2, d_reg=2)
    h = T([[[L3, 0.0], [0.0, 0.0]]])
    V = O.att_registers(arch, att_params(), h)[0]
    np.testing.assert_allclose(V.numpy(), [0.75 * L3, 0.0, 0.0, 0.5 * L3], rtol=0, atol=TOL)


def test_attention_jastrow_hand_case():
    """J_att = exp(MLP_1(V)) MLP_2(V) on V = [3/4 ln 3, 0, 0, 1/2 ln 3]:
    MLP_1 takes V_0 and V_3 (W1 picks them), W2 = I, b = 0, w3 = [1, 1];
    MLP_2 = 3/4 ln 3 - 7/8 ln 7 < 0 for every V."""
    arch = synth.Arch(width=2, n_layers=1, n_reg=2, d_reg=2)
    w1 = np.zeros((4, 2))
    w1[0, 0] = 1.0
    w1[3, 1] = 1.0
    p = dict(att_params())
    p.update({"ja1_w1": T(w1), "ja1_b1": T([0.0, 0.0]), "ja1_w2": T(np.eye(2)), "ja1_b2": T([0.0, 0.0]),
              "ja1_w3": T([1.0, 1.0]), "ja1_b3": T([0.0]),
              "ja2_w1": T(np.zeros((4, 2))), "ja2_b1": T([0.0, 0.0]), "ja2_w2": T(np.zeros((2, 2))),
              "ja2_b2": T([L3, L7]), "ja2_w3": T([1.0, -1.0]), "ja2_b3": T([0.0])})
    h = T([[[L3, 0.0], [0.0, 0.0]]])
    lj, sj = O.att_jastrow(arch, p, h)
    g1 = silu_closed(silu_closed(0.75 * L3)) + silu_closed(silu_closed(0.5 * L3))
    g2 = 0.75 * L3 - 0.875 * L7
    assert abs(float(lj[0]) - (g1 + math.log(abs(g2)))) < TOL
    assert float(sj[0]) == -1.0
