"""Autotuner of the moment pass (steps a2/a3): per degree L and precision it chooses the warp-tile
size (atoms per lane), the persistent grid's CTAs per SM and, for the mixed path, the
L-chunking (the float kernel's accumulator budget kmax: 160 or 96 per lane, which sets how many
column chunks the (L+1)^2 components take and how many CTAs fit on an SM) by timing the
caller's own batch.

For every degree present in the batch, the items of that degree (at most ``max_items_per_l`` of
them) form a sub-batch; each candidate setting (atoms per lane, CTAs per SM, kmax) is applied
with ``tcm_ctx_set_tiling_l`` and ``tcm_ctx_set_chunking_l``, the sub-batch is run once untimed
and ``reps`` times timed, and the median time of the moment phase (the library's CUDA-event
phase profile: the moment kernels of that degree, nothing else) is kept.  The fastest candidate
(when the sub-batch is a sample of the degree's items: among those within 1 % of it, the one
with the largest warp tiles; ``choose``) is applied to the context and returned.  Results can be saved to a JSON file keyed by device
name, library build and precision, and loaded into a later context.

The tiling and the chunking change only the order in which atom contributions are summed, so
every candidate gives results within the stated tolerances; the choice is made on time alone.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

DEFAULT_ATOMS_PER_LANE = (16, 32, 48, 64, 96, 128, 256)
DEFAULT_CTAS_PER_SM = (1, 2, 3)
DEFAULT_KMAX = (160, 96)  # the mixed path's chunk budgets (tcm_ctx_set_chunking_l)
FP64_KMAX = 80            # the double kernels' budget (fixed)


def ctas_limit(precision, kmax):
    """CTAs per SM the moment kernel of that precision and budget is compiled for."""
    from . import tcm
    if precision == tcm.TCM_FP64:
        return 2
    return 3 if kmax <= 96 else 2


def candidates(precision, atoms_per_lane=DEFAULT_ATOMS_PER_LANE, ctas_per_sm=DEFAULT_CTAS_PER_SM,
               kmax=DEFAULT_KMAX):
    """Every (atoms_per_lane, ctas_per_sm, kmax) the tuner times, in timing order."""
    from . import tcm
    kms = (FP64_KMAX,) if precision == tcm.TCM_FP64 else tuple(kmax)
    return [(a, c, k) for k in kms for a in atoms_per_lane for c in ctas_per_sm if c <= ctas_limit(precision, k)]


def get_setting(ctx, precision, L):
    from . import tcm
    apl, cps = ctx.tcm_ctx_get_tiling_l(precision, L)
    km = FP64_KMAX if precision == tcm.TCM_FP64 else ctx.tcm_ctx_get_chunking_l(L)[0]
    return (apl, cps, km)


def set_setting(ctx, precision, L, setting):
    from . import tcm
    apl, cps, km = setting
    ctx.tcm_ctx_set_tiling_l(precision, L, apl, cps)
    if precision != tcm.TCM_FP64:
        ctx.tcm_ctx_set_chunking_l(L, km)


@dataclass
class TuneResult:
    precision: int
    best: dict = field(default_factory=dict)     # L -> (atoms_per_lane, ctas_per_sm, kmax)
    timings: dict = field(default_factory=dict)  # L -> {(atoms_per_lane, ctas_per_sm, kmax): median ms}

    def to_json(self):
        return {"precision": int(self.precision),
                "best": {str(L): list(v) for L, v in self.best.items()},
                "timings": {str(L): {"x".join(str(x) for x in c): ms for c, ms in t.items()}
                            for L, t in self.timings.items()}}

    @classmethod
    def from_json(cls, d):
        r = cls(int(d["precision"]))
        r.best = {int(L): tuple(int(x) for x in v) for L, v in d["best"].items()}
        r.timings = {int(L): {tuple(int(x) for x in k.split("x")): float(ms) for k, ms in t.items()}
                     for L, t in d.get("timings", {}).items()}
        return r


def choose(timings: dict, tol=0.01):
    """Among the candidates within ``tol`` (relative) of the smallest median time, the one with
    the largest warp tiles (atoms per lane; ties: the first in candidate order).  Larger tiles
    mean fewer partial rows for the finalisation to read, which a sampled sub-batch
    under-represents: on the large assembly 256 and 512 atoms per lane time within 0.1 % on 512
    orientations, and 512 is 1.4 % faster on all 10,000.  ``tune`` passes tol = 0.01 when it
    timed a sample of a degree's items and 0 when it timed all of them."""
    if not timings:
        return None
    best_ms = min(timings.values())
    best = None
    for cand, ms in timings.items():
        if ms <= best_ms * (1.0 + tol) and (best is None or cand[0] > best[0]):
            best = cand
    return best


def degree_groups(lmax, max_items_per_l):
    """Indices of the items of each degree, at most max_items_per_l per degree (evenly strided)."""
    lmax = np.asarray(lmax)
    out = {}
    for L in sorted(set(int(x) for x in lmax)):
        idx = np.nonzero(lmax == L)[0]
        if len(idx) > max_items_per_l:
            idx = idx[np.linspace(0, len(idx) - 1, max_items_per_l).round().astype(int)]
        out[L] = idx
    return out


def moment_phase_ms(ctx, run, reps):
    """Median over reps of the moment-phase time of run() (one untimed call first)."""
    run()
    ctx.tcm_ctx_set_profiling(True)
    ctx.tcm_ctx_read_profile()
    times = []
    for _ in range(reps):
        run()
        ms, _ = ctx.tcm_ctx_read_profile()
        times.append(ms["moments"])
    ctx.tcm_ctx_set_profiling(False)
    return float(np.median(times))


def tune(ctx, systems, a, b, lmax, R0, rotB=None, precision=None, atoms_per_lane=DEFAULT_ATOMS_PER_LANE,
         ctas_per_sm=DEFAULT_CTAS_PER_SM, kmax=DEFAULT_KMAX, reps=3, max_items_per_l=512,
         measure=None) -> TuneResult:
    """Tune the moment pass on this batch (arguments as for ``Context.tcm_energy_batch``).

    ``measure(L, run) -> ms`` replaces the CUDA-event measurement (used by the host-side tests).
    The best setting per degree is applied to ``ctx`` before returning.
    """
    from . import tcm
    if precision is None:
        precision = tcm.TCM_MIXED
    a, b, lmax = np.asarray(a), np.asarray(b), np.asarray(lmax)
    R0 = np.asarray(R0, dtype=np.float64).reshape(-1, 3)
    rot = None if rotB is None else np.asarray(rotB, dtype=np.float64).reshape(-1, 3, 3)
    res = TuneResult(int(precision))
    for L, idx in degree_groups(lmax, max_items_per_l).items():
        pb = tcm.pack_batch(systems, a[idx], b[idx], lmax[idx], R0[idx], None if rot is None else rot[idx])

        def run(pb=pb):
            ctx.tcm_energy_batch_packed(pb, precision)

        default = get_setting(ctx, precision, L)
        t = {}
        for cand in candidates(precision, atoms_per_lane, ctas_per_sm, kmax):
            set_setting(ctx, precision, L, cand)
            t[cand] = measure(L, run) if measure else moment_phase_ms(ctx, run, reps)
        # a sub-batch that leaves out items of this degree under-represents the partial rows that
        # larger tiles save: then prefer them within 1 %; the whole batch is timed as it is
        subsampled = len(idx) < int(np.count_nonzero(lmax == L))
        best = choose(t, tol=0.01 if subsampled else 0.0) or default
        set_setting(ctx, precision, L, best)
        res.best[L] = best
        res.timings[L] = t
    return res


def apply(ctx, result: TuneResult):
    for L, setting in result.best.items():
        set_setting(ctx, result.precision, L, setting)


def library_key(lib_path=None, device_name=None):
    """Device name and a hash of the built library: a tuning is reused only on the same pair."""
    if lib_path is None:
        from . import tcm
        lib_path = tcm.LIB_PATH
    h = hashlib.sha256(open(lib_path, "rb").read()).hexdigest()[:16]
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    return f"{device_name}|{h}"


def save(path, result: TuneResult, key: str):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data.setdefault(key, {})[str(result.precision)] = result.to_json()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(ctx, path, precision, key: str):
    """Apply a saved tuning for (key, precision) if there is one; returns it or None."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    d = data.get(key, {}).get(str(int(precision)))
    if d is None:
        return None
    r = TuneResult.from_json(d)
    apply(ctx, r)
    return r
