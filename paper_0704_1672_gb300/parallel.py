"""Sharding over ranks (one process per GPU, torch.distributed).

Two kinds of work partition:

* independent items (orientations, pairs, requests): ``shard_items`` gives each rank a
  contiguous slice; nothing is exchanged (weak scaling of the benchmark, replicas);
* the moments of one system too large for one device: every rank takes a contiguous range
  of atoms (``shard_range``), the global centroid and radius come from one all-reduce of
  (sum x, sum y, sum z, n) and one max-all-reduce, every rank computes the moments of its
  atoms about that centre, and one all-reduce of the (Lmax+1)^2 doubles adds them up
  (Eq. (multipole) is a sum over atoms).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int):
    """Contiguous [lo, hi) of n units for this rank (the first n % world ranks get one more)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_items(n_items: int, rank: int, world: int):
    lo, hi = shard_range(n_items, rank, world)
    return np.arange(lo, hi)


def global_center_radius(xyz_local: torch.Tensor, group=None):
    """Centroid and radius of a system whose atoms are spread over the ranks (double)."""
    x = xyz_local.to(torch.float64)
    s = torch.zeros(4, dtype=torch.float64, device=x.device)
    if x.numel():
        s[:3] = x[:, :3].sum(0)
    s[3] = float(x.shape[0])
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    c = s[:3] / torch.clamp(s[3], min=1.0)
    r2 = torch.zeros(1, dtype=torch.float64, device=x.device)
    if x.numel():
        r2[0] = ((x[:, :3] - c) ** 2).sum(1).max()
    dist.all_reduce(r2, op=dist.ReduceOp.MAX, group=group)
    return c.cpu().numpy(), float(torch.sqrt(r2)[0])


def allreduce_moments(q: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the packed double moments of all ranks in place (the only exchange of the path)."""
    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return q


def sharded_moments(xyzq_local: torch.Tensor, lmax: int, moment_fn=None, group=None):
    """Moments of a system split over the ranks (this rank holds ``xyzq_local``).

    ``moment_fn(xyzq, lmax, center, radius) -> packed double tensor`` computes the moments of a
    set of atoms about a given centre; by default the library's tcm_moments on the current
    device (mixed precision).  Returns (packed moments, centre, radius), identical on all ranks.
    """
    c, a = global_center_radius(xyzq_local, group)
    if moment_fn is None:
        from . import tcm
        ctx = tcm.Context(lmax_cap=lmax)
        q = ctx.tcm_moments(xyzq_local, lmax, precision=tcm.TCM_MIXED, center=c, radius=a).q
        ctx.close()
    else:
        q = moment_fn(xyzq_local, lmax, c, a)
    q = q.to(torch.float64).contiguous()
    allreduce_moments(q, group)
    return q, c, a
