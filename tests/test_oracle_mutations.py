"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of an oracle function (a textual edit
of its source, executed in the oracle module's namespace and swapped in for
the duration of the test) and checks that the hand-worked pin of that
function now fails.  The planted mistakes are the ones a reader of the
Methods equations could plausibly make: swapped GLU operands, LayerNorm in
the wrong place, exp(-sigma x^2) for exp(-sigma^2 x^2), a missing log(1+r)/r
rescale, a reordered message concatenation, swapped spin channels, a missing
residual, a dropped readout layer, sum/log confusions in the Jastrow
readouts and a scaled attention softmax.
"""
import inspect
import textwrap

import pytest

from oracle import fire_oracle as O
import test_oracle_forward_pins as P

MUTATIONS = [
    ("glu", 'silu(y @ p["glu_wg"]) * (y @ p["glu_wv"])', 'silu(y @ p["glu_wv"]) * (y @ p["glu_wg"])',
     [P.test_glu_hand_case]),
    ("glu", 'y = layer_norm(x, p["ln_gamma"], p["ln_beta"])', 'y = x', [P.test_glu_hand_case]),
    ("glu", 'return (silu(y @ p["glu_wg"]) * (y @ p["glu_wv"])) @ p["glu_wo"]',
     'return (silu(y @ p["glu_wg"]) * (y @ p["glu_wv"])) @ p["glu_wo"].T', [P.test_glu_hand_case]),
    ("radial_filter", "torch.exp(-(sigma ** 2) * x0[..., None] ** 2)", "torch.exp(-sigma * x0[..., None] ** 2)",
     [P.test_radial_filter_hand_case]),
    ("radial_filter", "return g * (chi @ wenv)", "return g * (chi @ wenv.T)", [P.test_radial_filter_hand_case]),
    ("radial_filter", "g = silu(u) @ w2", "g = silu(u) @ w2.T",
     [P.test_radial_filter_hand_case]),
    ("radial_filter", 'u = torch.einsum("...mk,mkh->...mh", e, w1) + b1',
     'u = torch.einsum("...mk,mkh->...mh", e, w1.flip(0)) + b1.flip(0)', [P.test_radial_filter_per_nucleus_weights]),
    ("pair_features", "torch.log1p(sdist) / sdist", "1.0 / sdist", [P.test_pair_features_hand_case]),
    ("pair_features", "torch.log1p(sdist) / sdist", "torch.log1p(sdist)", [P.test_pair_features_hand_case]),
    ("en_sum", 'eb_en @ p["en_wfeat"]', 'e_en @ p["en_wfeat"]', [P.test_electron_nucleus_sum_hand_case]),
    ("en_sum", 'return (mask_en * gam * feat).sum(dim=2)', 'return (mask_en * gam * feat).mean(dim=2)',
     [P.test_electron_nucleus_sum_hand_case]),
    ("message_pass", "cat = torch.cat([h0[:, :, None, :].expand(B, n, n, h0.shape[-1]),\n"
                     "                     h0[:, None, :, :].expand(B, n, n, h0.shape[-1]), eb_ee], dim=-1)",
     "cat = torch.cat([h0[:, None, :, :].expand(B, n, n, h0.shape[-1]),\n"
     "                     h0[:, :, None, :].expand(B, n, n, h0.shape[-1]), eb_ee], dim=-1)",
     [P.test_message_pass_hand_case]),
    ("message_pass", "for alpha, sel in ((0, same), (1, ~same)):", "for alpha, sel in ((1, same), (0, ~same)):",
     [P.test_message_pass_hand_case]),
    ("message_pass", "msg = gam_ee * silu(z)", "msg = silu(gam_ee * z)", [P.test_message_pass_hand_case]),
    ("message_pass", "dee = r[:, :, None, :] - r[:, None, :, :]", "dee = r[:, None, :, :] - r[:, :, None, :]",
     [P.test_message_pass_hand_case]),
    ("embedding_mlp", 'h = h + silu(h @ p["mlp_w"][l] + p["mlp_b"][l])', 'h = silu(h @ p["mlp_w"][l] + p["mlp_b"][l])',
     [P.test_embedding_mlp_hand_case]),
    ("mlp_readout", 'a = silu(a @ p[pre + "_w2"] + p[pre + "_b2"])', 'a = a @ p[pre + "_w2"] + p[pre + "_b2"]',
     [P.test_mlp_readout_hand_case]),
    ("mlp_jastrow", 'f1 = mlp_readout(h, p, "jm1").sum(-1)', 'f1 = mlp_readout(h, p, "jm1").mean(-1)',
     [P.test_mlp_jastrow_hand_case]),
    ("mlp_jastrow", 'f2 = mlp_readout(h, p, "jm2").sum(-1)', 'f2 = mlp_readout(h, p, "jm2").prod(-1)',
     [P.test_mlp_jastrow_hand_case]),
    ("att_registers", "a = torch.softmax(scores, dim=-1)", "a = torch.softmax(scores / h.shape[-1] ** 0.5, dim=-1)",
     [P.test_attention_registers_hand_case]),
    ("att_registers", "a = torch.softmax(scores, dim=-1)", "a = torch.softmax(scores, dim=-2)",
     [P.test_attention_registers_hand_case]),
    ("att_jastrow", "return g1 + torch.log(torch.abs(g2)), torch.sign(g2)", "return g1 + g2, torch.sign(g2)",
     [P.test_attention_jastrow_hand_case]),
    ("att_jastrow", 'g2 = mlp_readout(V, p, "ja2")', 'g2 = mlp_readout(V, p, "ja1")',
     [P.test_attention_jastrow_hand_case]),
]


def _mutated(name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(O, name)))
    assert src.count(old) == 1, (name, old)
    ns = {}
    exec(compile(src.replace(old, new), f"<mutated {name}>", "exec"), O.__dict__, ns)
    return ns[name]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[f"{m[0]}-{i}" for i, m in enumerate(MUTATIONS)])
def test_planted_mistake_fails_a_pin(monkeypatch, name, old, new, pins):
    monkeypatch.setattr(O, name, _mutated(name, old, new))
    failed = 0
    for pin in pins:
        params = [m for m in getattr(pin, "pytestmark", []) if m.name == "parametrize"]
        cases = params[0].args[1] if params else [()]
        for case in cases:
            try:
                pin(*case) if params else pin()
            except (AssertionError, RuntimeError):
                failed += 1
    assert failed > 0, f"planted mistake in {name} passed every pin"


def test_unmutated_oracle_passes_the_pins():
    for _, _, _, pins in MUTATIONS:
        for pin in pins:
            params = [m for m in getattr(pin, "pytestmark", []) if m.name == "parametrize"]
            for case in (params[0].args[1] if params else [()]):
                pin(*case) if params else pin()
