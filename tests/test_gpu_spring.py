"""GPU parity of fire_spring_step (Methods, "Variational Monte Carlo",
eq. spring) with the FP64 oracle.

The Gram matrix comes from the tensor cores, which accumulate each chunk of
4096 parameters in float32 with an error of about 2^-22 of the running sum
per 16-deep step (a systematic, not a random-walk, growth: measured 2.8e-5
of sqrt(G_ii G_jj) over 188 steps); the chunks are summed and centred in
float64.  Bounds: per entry of the centred Gram matrix
|dK_ij| <= s 2^-22 (r_i r_j + r_i m + r_j m + m^2), s the 16-deep steps of a
chunk, r_i = |O_i| and m = mean r (the centring P G P passes the row and
column means of the error on); delta to 2e-3 of its largest entry with the
damping 0.1 mean diag K (condition number below 11).  At the C26H24 workload
(4096 walkers' gradient rows and local energies from the library itself, 5.1 M
parameters) the oracle cannot form the product, so sampled Gram entries are
checked against float64 dot products of the two rows, the solve against its
own residual in float64, and sampled entries of delta against
sum_i Obar_ip x_i + eta delta_prev,p."""
import numpy as np
import pytest
import torch

from oracle import spring_oracle as S
from paper_2504_06087_gb300 import fire, synth

pytestmark = pytest.mark.gpu


def _rows(N, P, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    scale = torch.exp(torch.randn(P, generator=g, dtype=torch.float64) * 1.5)
    O = (torch.randn(N, P, generator=g, dtype=torch.float64) * scale + 0.3 * scale).float()
    e = torch.randn(N, generator=g, dtype=torch.float64) * 3.0 - 120.0
    d0 = (torch.randn(P, generator=g, dtype=torch.float64) * 1e-3).float()
    return O, e, d0


CHUNK = 4096


def gram_bound(rn, P):
    """Entrywise bound of the centred Gram error (module docstring)."""
    steps = min((P + 63) // 64 * 64, CHUNK) / 16
    m = rn.mean()
    return steps * 2.0 ** -22 * (np.outer(rn, rn) + (rn[:, None] + rn[None, :]) * m + m * m)


@pytest.mark.parametrize("N,P,eta,with_prev", [(64, 3001, 0.99, True), (200, 5000, 0.0, False),
                                               (32, 60_000, 0.99, True)])
def test_spring_matches_oracle(N, P, eta, with_prev):
    O, e, d0 = _rows(N, P, N + P)
    Od = O.double().numpy()
    lam = 0.1 * float(((Od - Od.mean(0)) ** 2).sum(1).mean())
    ref_d, ref_K, ref_x = S.spring_update(Od, e.numpy(), d0.double().numpy() if with_prev else None, eta, lam)
    out = fire.spring_step(O.cuda(), e.cuda(), d0.cuda() if with_prev else None, eta, lam, want_gram=True,
                           want_x=True)
    K = out["gram"].cpu().numpy()
    bound = gram_bound(np.linalg.norm(Od, axis=1), P)
    assert np.all(np.abs(K - ref_K) <= bound), np.max(np.abs(K - ref_K) / bound)
    d = out["delta"].double().cpu().numpy()
    assert np.max(np.abs(d - ref_d)) < 2e-3 * np.max(np.abs(ref_d))


def test_spring_momentum_fixed_point_on_gpu():
    """eps = eta Obar delta_prev (plus a constant) leaves delta = eta delta_prev."""
    O, _, d0 = _rows(48, 4000, 5)
    Od = O.double()
    Ob = Od - Od.mean(0)
    eta = 0.99
    e = eta * (Ob @ d0.double()) + 11.0
    lam = 1e-3 * float(Ob.pow(2).sum(1).mean())
    out = fire.spring_step(O.cuda(), e.cuda(), d0.cuda(), eta, lam)
    d = out["delta"].double().cpu()
    assert float((d - eta * d0.double()).abs().max()) < 1e-4 * float((eta * d0.double()).abs().max())


def test_spring_rejects_bad_arguments():
    O = torch.zeros(4, 10, device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert fire.spring_step(O, e, None, 0.9, 0.0, check=False)["status"] == 1
    assert fire.spring_step(O, e, None, -1.0, 1e-3, check=False)["status"] == 1
    with pytest.raises(fire.FireError):       # one walker: no workspace size, rejected on the host
        fire.spring_step(O[:1], e[:1], None, 0.9, 1e-3)


def test_spring_on_c26h24_gradient_rows():
    """One SPRING step on the C26H24 workload: 4096 walkers' gradient rows
    (float32, 5.1 M parameters) and local energies from the library itself."""
    w = synth.workload("c26h24")
    r, p = synth.make_inputs(w, 4096)
    f = fire.Fire(w.system, w.arch, p, "fp32")
    rt = torch.as_tensor(r, device=f.device)
    O = f.grad_logpsi(rt)["grad"]
    del f
    torch.cuda.empty_cache()
    fb = fire.Fire(w.system, w.arch, p, "bf16")
    e = fb.local_energy(rt)["e_loc"]
    del fb
    torch.cuda.empty_cache()
    N, P = O.shape
    d0 = torch.zeros(P, dtype=torch.float32, device=O.device)
    d0[::97] = 1e-4
    eta = 0.99
    out = fire.spring_step(O, e, d0, eta, 1e-3, want_gram=True, want_x=True)
    K, x = out["gram"], out["x"]
    rng = np.random.default_rng(9)
    Ocpu_rows = {}

    def row(i):
        if i not in Ocpu_rows:
            Ocpu_rows[i] = O[i].double().cpu().numpy()
        return Ocpu_rows[i]

    # column means and the projection O d0 in float64, 256 rows at a time
    cm = np.zeros(P)
    od = torch.empty(N, dtype=torch.float64, device=O.device)
    for i0 in range(0, N, 256):
        blk = O[i0:i0 + 256].double()
        cm += blk.sum(0).cpu().numpy()
        od[i0:i0 + 256] = blk @ d0.double()
        del blk
    cm /= N
    rn = torch.cat([O[i0:i0 + 256].double().pow(2).sum(1).sqrt() for i0 in range(0, N, 256)]).cpu().numpy()
    for _ in range(12):
        i, j = (int(v) for v in rng.integers(0, N, 2))
        kij = float(np.dot(row(i) - cm, row(j) - cm))
        m = rn.mean()
        bound = CHUNK / 16 * 2.0 ** -22 * (rn[i] * rn[j] + (rn[i] + rn[j]) * m + m * m)
        assert abs(float(K[i, j]) - kij) <= bound, (i, j, float(K[i, j]), kij, bound)
    # the solve: (K + lambda I) x = eps - eta Obar d0, residual in float64
    Kd = K.clone()
    Kd.diagonal().add_(1e-3)
    eps = e - e.mean()
    od0 = od - float(np.dot(cm, d0.double().cpu().numpy()))
    b = eps - eta * od0
    # backward stability of the float64 Cholesky solve: the residual is a
    # rounding-level multiple of |K| |x|
    res = (Kd @ x - b).abs().max() / (Kd.abs().max() * x.abs().sum() + b.abs().max())
    assert float(res) < 1e-12, float(res)
    # sampled entries of delta
    xs = x.cpu().numpy()
    for pcol in rng.integers(0, P, 16):
        col = O[:, int(pcol)].double().cpu().numpy()
        want = float(np.dot(col - cm[pcol], xs)) + eta * float(d0[int(pcol)])
        got = float(out["delta"][int(pcol)])
        assert abs(got - want) <= 1e-5 * max(abs(want), 1e-30) + 1e-30, (pcol, got, want)
