"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a special case that reduces to a textbook result, or finite
differences, chosen so that a dropped term, a wrong sign or a swapped operand
in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import torch

from paper_2504_06087_gb300 import synth
from oracle import fire_oracle as O
from recipes import const_h_params


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

def test_fcut_is_c2_and_vanishes_beyond_cutoff():
    # p = 6: u'(s) = -168 s^5 (1 - s)^2, derived by hand from the polynomial.
    s = torch.linspace(0.0, 1.3, 131, dtype=torch.float64, requires_grad=True)
    u = O.f_cut(s)
    (du,) = torch.autograd.grad(u.sum(), s, create_graph=True)
    (d2u,) = torch.autograd.grad(du.sum(), s)
    sd = s.detach()
    ref = torch.where(sd < 1, -168 * sd ** 5 * (1 - sd) ** 2, torch.zeros_like(sd))
    assert torch.allclose(du.detach(), ref, atol=1e-12)
    assert float(u[0].detach()) == 1.0
    assert torch.all(u.detach()[sd >= 1.0] == 0.0)
    near = (sd > 0.999) & (sd < 1.0)
    assert torch.all(u.detach()[near].abs() < 1e-12)
    assert torch.all(d2u[near].abs() < 1e-3)


def test_layer_norm_matches_library():
    x = torch.randn(7, 33, dtype=torch.float64)
    g, b = torch.randn(33, dtype=torch.float64), torch.randn(33, dtype=torch.float64)
    ref = torch.nn.functional.layer_norm(x, (33,), g, b, eps=O.LN_EPS)
    assert torch.allclose(O.layer_norm(x, g, b), ref, atol=1e-13)


def test_silu_derivatives_closed_form():
    x = torch.linspace(-6, 6, 101, dtype=torch.float64, requires_grad=True)
    y = O.silu(x)
    (d1,) = torch.autograd.grad(y.sum(), x, create_graph=True)
    (d2,) = torch.autograd.grad(d1.sum(), x)
    s = torch.sigmoid(x.detach())
    xd = x.detach()
    assert torch.allclose(d1.detach(), s * (1 + xd * (1 - s)), atol=1e-14)
    assert torch.allclose(d2, s * (1 - s) * (2 + xd * (1 - 2 * s)), atol=1e-14)


# ---------------------------------------------------------------------------
# closed forms of the local energy
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("sigma,z", [(1.0, 1.0), (0.7, 1.0), (1.3, 2.0)])
def test_hydrogen_like_closed_form(sigma, z):
    """Psi = exp(-sigma r) on a charge-Z nucleus: E_L = -sigma^2/2 + (sigma - Z)/r."""
    system = synth.System(np.zeros((1, 3)), np.array([z]), 1, 1, 5.0, 20.0, "H")
    arch = synth.Arch(width=8, n_layers=1, n_det=1, n_env=1, jastrow_width=8, flags=0)
    p = const_h_params(system, arch)
    p["orb_w"][:] = 1.0
    p["env_pi"][:] = 1.0
    p["env_sigma"][:] = sigma
    r = np.random.default_rng(0).standard_normal((6, 1, 3)) * 1.5
    e, la, sg = O.local_energy(system, arch, p, r)
    rr = np.linalg.norm(r[:, 0], axis=-1)
    ref = -sigma ** 2 / 2 + (sigma - z) / rr
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-12)
    if sigma == 1.0 and z == 1.0:
        np.testing.assert_allclose(e, -0.5, atol=1e-12)


def test_two_electron_product_closed_form():
    """1 up + 1 down electron, diagonal orbital matrix of two exponentials:
    E_L = sum_i (-s_i^2/2 + (s_i - Z)/r_i) + 1/r_12."""
    z, s0, s1 = 2.0, 1.6, 0.9
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
    r = np.random.default_rng(1).standard_normal((5, 2, 3))
    e, _, _ = O.local_energy(system, arch, p, r)
    r0, r1 = np.linalg.norm(r[:, 0], axis=-1), np.linalg.norm(r[:, 1], axis=-1)
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=-1)
    ref = (-s0 ** 2 / 2 + (s0 - z) / r0) + (-s1 ** 2 / 2 + (s1 - z) / r1) + 1 / r12
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-11)


def test_potential_by_hand():
    system = synth.water()
    # nuclear repulsion of water, numbers written out
    rep = 8 * 1 / 1.81 + 8 * 1 / math.sqrt(0.45 ** 2 + 1.75 ** 2) \
        + 1 * 1 / math.sqrt((1.81 + 0.45) ** 2 + 1.75 ** 2)
    r = np.zeros((1, 10, 3))
    r[0, :, 0] = np.arange(10) * 3.0 + 100.0       # electrons on a far line
    r[0, :, 1] = 7.0
    v = O.potential(system, torch.as_tensor(r)).item()
    ee = sum(1.0 / (3.0 * (j - i)) for i in range(10) for j in range(i + 1, 10))
    en = 0.0
    for i in range(10):
        x, y = 100.0 + 3.0 * i, 7.0
        en -= 8 / math.hypot(x, y) + 1 / math.hypot(x - 1.81, y) + 1 / math.hypot(x + 0.45, y - 1.75)
    assert abs(v - (rep + ee + en)) < 1e-12


def test_cusp_jastrow_satisfies_kato_cusp():
    """d/dr of the pair term at r -> 0 is -w: 1/2 (anti) and 1/4 (parallel) at init."""
    system = synth.System(np.zeros((1, 3)), np.array([2.0]), 3, 2, 5.0, 20.0, "x")
    p = O.params_to_torch(synth.init_params(system, synth.Arch(width=8, n_layers=1, n_det=1), 0))
    for (a, b), want in (((0, 2), 0.5), ((0, 1), 0.25)):
        eps = 1e-7
        base = np.array([[[0.0, 0.0, 0.0], [1e6, 0.0, 0.0], [0.0, 1e6, 0.0]]])
        r1, r2 = base.copy(), base.copy()
        r1[0, b] = r1[0, a] + [eps, 0, 0]
        r2[0, b] = r2[0, a] + [2 * eps, 0, 0]
        j1 = O.cusp_jastrow(system, p, torch.as_tensor(r1)).item()
        j2 = O.cusp_jastrow(system, p, torch.as_tensor(r2)).item()
        assert abs((j2 - j1) / eps - want) < 1e-5


# ---------------------------------------------------------------------------
# invariants and derivatives of the full ansatz
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def water_case():
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 4)
    return w, r, p


def test_laplacian_and_gradient_match_finite_differences(water_case):
    w, r, p = water_case
    r = r[:2]
    e, la, sg, kin, v, g, lap = O.local_energy(w.system, w.arch, p, r, return_parts=True)
    n = w.system.n_el
    for b in range(r.shape[0]):
        f0 = O.logpsi_np(w.system, w.arch, p, r[b:b + 1])[0][0]

        def second(hh):
            pts = []
            for i in range(n):
                for x in range(3):
                    for s in (1, -1):
                        q = r[b].copy()
                        q[i, x] += s * hh
                        pts.append(q)
            vals = O.logpsi_np(w.system, w.arch, p, np.stack(pts))[0].reshape(n, 3, 2)
            return (vals[..., 0] - 2 * f0 + vals[..., 1]) / hh ** 2, (vals[..., 0] - vals[..., 1]) / (2 * hh)

        d1, g1 = second(2e-3)
        d2, g2 = second(1e-3)
        rich = (4 * d2 - d1) / 3
        grich = (4 * g2 - g1) / 3
        assert abs(rich.sum() - lap[b]) <= 1e-7 * max(1.0, abs(lap[b]))
        np.testing.assert_allclose(grich, g[b], rtol=0, atol=1e-8 * max(1.0, np.abs(g[b]).max()))


def test_antisymmetry_same_spin_exchange(water_case):
    w, r, p = water_case
    e0, la0, s0 = O.local_energy(w.system, w.arch, p, r)
    for (a, b) in ((0, 3), (6, 9)):              # two up, two down electrons
        q = r.copy()
        q[:, [a, b]] = q[:, [b, a]]
        e1, la1, s1 = O.local_energy(w.system, w.arch, p, q)
        np.testing.assert_array_equal(s1, -s0)
        np.testing.assert_allclose(la1, la0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(e1, e0, rtol=1e-10, atol=1e-10)


def test_opposite_spin_exchange_is_not_a_symmetry(water_case):
    w, r, p = water_case
    q = r.copy()
    q[:, [0, 7]] = q[:, [7, 0]]
    la0, _ = O.logpsi_np(w.system, w.arch, p, r)
    la1, _ = O.logpsi_np(w.system, w.arch, p, q)
    assert np.max(np.abs(la1 - la0)) > 1e-3


def test_translation_invariance(water_case):
    w, r, p = water_case
    shift = np.array([0.37, -1.2, 2.5])
    sys2 = synth.System(w.system.nuc_pos + shift, w.system.nuc_charge, w.system.n_el,
                        w.system.n_up, w.system.cutoff, w.system.cutoff_nuc)
    e0, la0, s0 = O.local_energy(w.system, w.arch, p, r)
    e1, la1, s1 = O.local_energy(sys2, w.arch, p, r + shift)
    np.testing.assert_array_equal(s0, s1)
    np.testing.assert_allclose(la1, la0, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(e1, e0, rtol=1e-9, atol=1e-9)


def test_embedding_locality_is_exact():
    """h_i is bit-identical when an electron that stays beyond c of i moves."""
    w = synth.workload("c8h10")
    r, p = synth.make_inputs(w, 1)
    pt = O.params_to_torch(p)
    c = w.system.cutoff
    rr = r[0]
    d = np.linalg.norm(rr[:, None] - rr[None], axis=-1)
    k = 0
    q = rr.copy()
    q[k] += np.array([0.3, -0.2, 0.1])
    dq = np.linalg.norm(q[:, None] - q[None], axis=-1)
    far = [i for i in range(w.system.n_el) if i != k and d[i, k] > c and dq[i, k] > c]
    near = [i for i in range(w.system.n_el) if i != k and d[i, k] < c - 0.5]
    assert len(far) > 10 and len(near) > 0
    with torch.no_grad():
        h0a, h1a, ha = O.embeddings(w.system, w.arch, pt, torch.as_tensor(rr[None]))
        h0b, h1b, hb = O.embeddings(w.system, w.arch, pt, torch.as_tensor(q[None]))
    for i in far:
        assert torch.equal(ha[0, i], hb[0, i]) and torch.equal(h1a[0, i], h1b[0, i])
    # h^0 depends on the electron's own position only
    others = [i for i in range(w.system.n_el) if i != k]
    assert torch.equal(h0a[0, others], h0b[0, others])
    assert not torch.equal(ha[0, near[0]], hb[0, near[0]])


def test_cutoff_zero_reduces_to_slater_formula():
    """c = 0: rows of Phi depend on their own electron only, so
    Lap log det = sum_i [ sum_l Lap(Phi_il) A_li - sum_x (sum_l d_ix Phi_il A_li)^2 ]."""
    system = synth.zigzag_polyene(2, cutoff=0.0)
    arch = synth.Arch(width=16, n_layers=2, n_det=1, jastrow_width=16, flags=0)
    p = synth.init_params(system, arch, 7)
    r = synth.walkers(system, 2, 77)
    e, la, sg, kin, v, g, lap = O.local_energy(system, arch, p, r, return_parts=True)
    pt = O.params_to_torch(p)
    n = system.n_el
    for b in range(2):
        rb = torch.as_tensor(r[b:b + 1]).clone()
        with torch.no_grad():
            _, _, h = O.embeddings(system, arch, pt, rb)
            phi = O.orbitals(system, arch, pt, rb, h)[0, 0]
        A = torch.linalg.inv(phi)
        total = 0.0
        for i in range(n):
            def row(ri):
                q = rb.clone()
                q[0, i] = ri
                _, _, hh = O.embeddings(system, arch, pt, q)
                return O.orbitals(system, arch, pt, q, hh)[0, 0, i]
            x0 = rb[0, i].clone()
            jac = torch.autograd.functional.jacobian(row, x0)          # [n, 3]
            hes = torch.autograd.functional.hessian(lambda z: (row(z) * A[:, i]).sum(), x0)
            lapterm = torch.trace(hes)
            total += float(lapterm) - float(((jac * A[:, i, None]).sum(0) ** 2).sum())
        assert abs(total - lap[b]) < 1e-9 * max(1.0, abs(total))


def test_slogdet_matches_lapack(water_case):
    w, r, p = water_case
    pt = O.params_to_torch(p)
    with torch.no_grad():
        _, _, h = O.embeddings(w.system, w.arch, pt, torch.as_tensor(r))
        phi = O.orbitals(w.system, w.arch, pt, torch.as_tensor(r), h).numpy()
    s_np, l_np = np.linalg.slogdet(phi)
    la, sg, (s_o, l_o) = O.slater_part(w.system, w.arch, pt, torch.as_tensor(r), h)
    np.testing.assert_array_equal(s_o.numpy(), s_np)
    np.testing.assert_allclose(l_o.numpy(), l_np, rtol=1e-12)
    # the signed sum over determinants, written out with numpy
    tot = (s_np * np.exp(l_np)).sum(axis=1)
    np.testing.assert_allclose(la.detach().numpy(), np.log(np.abs(tot)), rtol=1e-12)
    np.testing.assert_array_equal(sg.detach().numpy(), np.sign(tot))


def test_attention_registers_uniform_special_case():
    """All embeddings equal => the softmax is uniform and v_r = h W^V_r."""
    arch = synth.Arch(width=16, n_layers=1, n_det=1, n_reg=3, d_reg=4)
    system = synth.water()
    p = O.params_to_torch(synth.init_params(system, arch, 3))
    hrow = torch.randn(16, dtype=torch.float64)
    h = hrow.expand(2, 10, 16)
    V = O.att_registers(arch, p, h)
    ref = torch.einsum("k,rkc->rc", hrow, p["att_wv"]).reshape(-1)
    assert torch.allclose(V[0], ref, atol=1e-13) and torch.allclose(V[1], ref, atol=1e-13)
    # and V is invariant under any permutation of electrons
    h2 = torch.randn(1, 10, 16, dtype=torch.float64)
    perm = torch.randperm(10)
    assert torch.allclose(O.att_registers(arch, p, h2), O.att_registers(arch, p, h2[:, perm]), atol=1e-13)


def test_parameter_gradient_matches_finite_differences(water_case):
    w, r, p = water_case
    r = r[:2]
    rng = np.random.default_rng(5)
    spec = synth.param_spec(w.system, w.arch)
    sizes = np.array([int(np.prod(s)) for _, s in spec])
    flat = rng.choice(sizes.sum(), size=64, replace=False)
    bounds = np.cumsum(sizes)
    picks = []
    for f in flat:
        k = int(np.searchsorted(bounds, f, side="right"))
        picks.append((spec[k][0], int(f - (bounds[k] - sizes[k]))))
    grads = O.grad_logpsi(w.system, w.arch, p, r, names=sorted({n for n, _ in picks}))
    hstep = 1e-4
    for name, idx in picks:
        pp, pm = {k: v.copy() for k, v in p.items()}, {k: v.copy() for k, v in p.items()}
        pp[name].reshape(-1)[idx] += hstep
        pm[name].reshape(-1)[idx] -= hstep
        fd = (O.logpsi_np(w.system, w.arch, pp, r)[0] - O.logpsi_np(w.system, w.arch, pm, r)[0]) / (2 * hstep)
        ad = grads[name].reshape(r.shape[0], -1)[:, idx]
        np.testing.assert_allclose(ad, fd, rtol=1e-6, atol=1e-7)
