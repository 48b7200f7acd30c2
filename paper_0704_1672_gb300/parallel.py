"""Sharding over ranks (one process per GPU, torch.distributed).

Two kinds of work partition:

* independent items (orientations, pairs, requests): ``shard_items`` gives each rank a
  contiguous slice; nothing is exchanged (weak scaling of the benchmark, replicas);
* the moments of one system too large for one device: every rank takes a contiguous range
  of atoms (``shard_range``); the library's step a1 gives each rank's coordinate sums, one
  all-reduce gives the global centroid, the library's radius about it and one max-all-reduce
  the global radius; every rank computes the moments of its atoms about that centre with the
  library, and one all-reduce of the (Lmax+1)^2 doubles adds them up (Eq. (multipole) is a sum
  over atoms).
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


def shard_center_sums(ctx, xyzq_local: torch.Tensor):
    """(sum x, sum y, sum z, n) of this rank's atoms, from the library's centroid (step a1 on the
    device): n times the shard's centroid."""
    n = int(xyzq_local.shape[0])
    if n == 0:
        return np.zeros(4)
    c, _ = ctx.tcm_prepare(xyzq_local)
    return np.array([c[0] * n, c[1] * n, c[2] * n, float(n)])


def shard_radius(ctx, xyzq_local: torch.Tensor, center) -> float:
    """Largest distance of this rank's atoms from the given (global) centre (step a1 on the device)."""
    if int(xyzq_local.shape[0]) == 0:
        return 0.0
    _, a = ctx.tcm_prepare(xyzq_local, center=center)
    return float(a)


def shard_moments(ctx, xyzq_local: torch.Tensor, lmax: int, center, radius, precision=None) -> torch.Tensor:
    """Moments of this rank's atoms about the global centre, scaled by the global radius
    (tcm_moments): their sum over the ranks is the system's moments."""
    from . import tcm
    precision = tcm.TCM_MIXED if precision is None else precision
    return ctx.tcm_moments(xyzq_local, lmax, precision=precision, center=center, radius=radius).q


def allreduce_moments(q: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the packed double moments of all ranks in place (the only exchange of the path)."""
    dist.all_reduce(q, op=dist.ReduceOp.SUM, group=group)
    return q


def global_center_radius(ctx, xyzq_local: torch.Tensor, group=None, geom=None):
    """Centroid and radius of a system whose atoms are spread over the ranks: each rank's
    coordinate sums and, about the resulting centre, its largest distance, from the library
    (``geom`` = (center_sums_fn, radius_fn) replaces it, e.g. on CPU ranks), combined by one
    sum-all-reduce and one max-all-reduce."""
    csum, rad = geom if geom is not None else (lambda x: shard_center_sums(ctx, x),
                                              lambda x, c: shard_radius(ctx, x, c))
    s = torch.tensor(csum(xyzq_local), dtype=torch.float64)
    dev_t = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    s = s.to(dev_t)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    s = s.cpu().numpy()
    c = s[:3] / max(s[3], 1.0)
    r = torch.tensor([rad(xyzq_local, c)], dtype=torch.float64, device=dev_t)
    dist.all_reduce(r, op=dist.ReduceOp.MAX, group=group)
    return c, float(r.cpu()[0])


def sharded_moments(xyzq_local: torch.Tensor, lmax: int, moment_fn=None, geom=None, group=None, precision=None):
    """Moments of a system split over the ranks (this rank holds ``xyzq_local``).

    The global centre and radius come from the library's step a1 on every rank's atoms plus two
    all-reduces; ``moment_fn(xyzq, lmax, center, radius) -> packed double tensor`` computes the
    moments of a set of atoms about a given centre, by default the library's tcm_moments on the
    current device.  ``geom`` and ``moment_fn`` stand in for the library on CPU ranks.  Returns
    (packed moments, centre, radius), identical on all ranks.
    """
    ctx = None
    if geom is None or moment_fn is None:
        from . import tcm
        ctx = tcm.Context(lmax_cap=lmax)
    try:
        c, a = global_center_radius(ctx, xyzq_local, group, geom)
        if moment_fn is None:
            q = shard_moments(ctx, xyzq_local, lmax, c, a, precision)
        else:
            q = moment_fn(xyzq_local, lmax, c, a)
    finally:
        if ctx is not None:
            ctx.close()
    q = q.to(torch.float64).contiguous()
    allreduce_moments(q, group)
    return q, c, a
