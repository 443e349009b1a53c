"""GPU parity of fire_ecp_nonlocal with the FP64 pseudopotential oracle
(oracle/ecp_oracle.py, full recompute of every ratio).

Tolerances per walker, relative to the magnitude of the summed terms
S = sum_kq |v_l(2l+1) w_q P_l ratio| (the oracle's scale; a rounding error
of a sum is relative to its summands, and the terms cancel): FP64 state
1e-10 S, float32 state 1e-4 S (the ratios carry the float32 rounding of the
low-rank update, as in the sampler).  Closed form: a spherical wave function around
the pseudopotential nucleus keeps only the s channel, V = v_0(|r - R|)."""
import numpy as np
import pytest

from oracle import ecp_oracle as E
from paper_2504_06087_gb300 import fire, synth
from recipes import hydrogen_like

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_hydrogen_s_channel_closed_form(prec, tol):
    system, arch, p = hydrogen_like(1.0, 1.0, width=32)
    ent = [{"n_quad": 12, "r_cut": 3.0, "terms": [[(3.0, 0, 1.5), (-1.0, 2, 0.7)], [(5.0, 1, 2.0)], [(2.0, 0, 0.9)]]}]
    r = np.random.default_rng(4).standard_normal((64, 1, 3))
    out = fire.Fire(system, arch, p, prec, k_cap=4).ecp_nonlocal(r, ent, seed=9)
    rad = np.linalg.norm(r[:, 0], axis=-1)
    want = np.where(rad < 3.0, 3.0 * np.exp(-1.5 * rad ** 2) - rad ** 2 * np.exp(-0.7 * rad ** 2), 0.0)
    assert rel(out["v_nl"].cpu().numpy(), want).max() < tol


WATER_ECP = [{"n_quad": 6, "r_cut": 1.5, "terms": [[(3.0, 0, 1.2), (-1.0, 2, 0.5)], [(2.0, 0, 0.8)]]}, None, None]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_water_matches_oracle(prec, tol):
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 16)
    ref, scale = E.nonlocal_energy(w.system, w.arch, p, r, WATER_ECP, seed=31, return_scale=True)
    assert np.count_nonzero(ref) >= 12
    out = fire.Fire(w.system, w.arch, p, prec).ecp_nonlocal(r, WATER_ECP, seed=31)
    err = np.abs(out["v_nl"].cpu().numpy() - ref)
    assert np.all(err <= tol * np.maximum(scale, 1e-300)), (err / scale).max()


def test_c8h10_tetrahedral_quadrature_matches_oracle():
    """Pseudopotentials on the eight carbons (N_quad = 4, r_cut 1.2 bohr, half
    the C-C distance is 1.3), s and d channels; float64 state."""
    w = synth.workload("c8h10")
    r, p = synth.make_inputs(w, 4)
    ecp = [{"n_quad": 4, "r_cut": 1.2, "terms": [[(4.0, 0, 1.0)], [], [(1.5, 0, 0.6)]]} if z == 6.0 else None
           for z in w.system.nuc_charge]
    ref, scale = E.nonlocal_energy(w.system, w.arch, p, r, ecp, seed=77, return_scale=True)
    out = fire.Fire(w.system, w.arch, p, "fp64").ecp_nonlocal(r, ecp, seed=77)
    err = np.abs(out["v_nl"].cpu().numpy() - ref)
    assert np.all(err <= 1e-10 * scale), (err / scale).max()


def test_bad_tables_are_rejected_on_the_host():
    w = synth.workload("water")
    r, p = synth.make_inputs(w, 2)
    f = fire.Fire(w.system, w.arch, p, "fp64")
    for bad in ({"n_quad": 5, "r_cut": 1.0, "terms": [[(1.0, 0, 1.0)]]},
                {"n_quad": 4, "r_cut": -1.0, "terms": [[(1.0, 0, 1.0)]]},
                {"n_quad": 4, "r_cut": 1.0, "terms": [[(1.0, 0, -2.0)]]}):
        assert f.ecp_nonlocal(r, [bad, None, None], check=False)["status"] == 1
