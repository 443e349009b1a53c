"""Walker sharding across GPUs (one process per GPU).

Walkers are independent: every entry point of the library evaluates a batch of
walkers with no data from other walkers, so N GPUs run N replicas, each on its
own contiguous block of the global walker range.  The only cross-rank step of
a variational Monte Carlo iteration that touches this path is the energy
estimate: one float64 all-reduce of (sum E_L, sum E_L^2, number of finite
E_L) per step.  Walkers on a node (E_L = NaN, a legitimate outcome) are left
out of the moments and counted.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch


def walker_block(n_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(first walker, count) of rank's contiguous block; the first
    n_total % world ranks take one walker more."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def energy_moments(e_loc: torch.Tensor, group: Optional[object] = None) -> dict:
    """Global mean and variance of E_L over every rank's walkers.

    e_loc: this rank's [W] local energies (any device; reduced in float64).
    Without an initialised process group the moments are the local ones."""
    e = e_loc.detach().to(torch.float64)
    ok = torch.isfinite(e)
    v = torch.stack([torch.where(ok, e, torch.zeros_like(e)).sum(),
                     torch.where(ok, e * e, torch.zeros_like(e)).sum(),
                     ok.sum().to(torch.float64),
                     (~ok).sum().to(torch.float64)])
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    s, s2, n, bad = (float(x) for x in v.cpu())
    mean = s / n if n > 0 else float("nan")
    var = max(s2 / n - mean * mean, 0.0) if n > 0 else float("nan")
    return {"mean": mean, "variance": var, "n": int(n), "n_nonfinite": int(bad)}
