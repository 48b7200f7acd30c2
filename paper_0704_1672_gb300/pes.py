"""Potential-energy-surface scan (Section IV): two systems fixed in space, the centre of B moved
over a grid of separations R0, the TCM energy at several Lmax and the exact Coulomb energy at
every grid point, and the relative error of Eq. (error),

    eta(Lmax)(R0) = |U_coul(R0) - U_mult^Lmax(R0)| / |U_coul(R0)| x 100 %.

The moments of A and B are computed once at the largest Lmax and kept on the device; every grid
point and every Lmax is then one item of a batched contraction (the moments are taken into the
frame of each R0 inside the contraction kernel), and the exact energies come from the batched
direct-sum kernel.  Everything runs in the library's kernels; the error map is arithmetic on the
results.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import time

import numpy as np


@dataclass
class PesResult:
    R0: np.ndarray                 # (n, 3) grid separations
    lmax: tuple
    U_mult: dict                   # Lmax -> (n,) TCM energies
    U_coul: np.ndarray | None      # (n,) exact energies, or None
    timings_ms: dict = field(default_factory=dict)

    def eta(self, L):
        """Eq. (error) in percent at every grid point."""
        return np.abs(self.U_coul - self.U_mult[L]) / np.abs(self.U_coul) * 100.0


def scan(ctx, A, B, R0, lmax_values, precision=None, direct=True, cA=None, cB=None):
    """TCM energies at every Lmax in ``lmax_values`` and (``direct``) exact energies at every
    separation in ``R0`` (n, 3), for device systems A and B (N, 4) in fixed orientations."""
    import torch

    from . import tcm
    if precision is None:
        precision = tcm.TCM_MIXED
    R0 = np.ascontiguousarray(R0, dtype=np.float64).reshape(-1, 3)
    n = len(R0)
    lmax_values = tuple(int(L) for L in lmax_values)
    Lhi = max(lmax_values)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    stream = torch.cuda.current_stream()
    ev[0].record(stream)
    mA = ctx.tcm_moments(A, Lhi, precision=precision, center=cA)
    mB = ctx.tcm_moments(B, Lhi, precision=precision, center=cB)
    systems = [tcm.make_system(A, mA.center, mA.radius, moments=mA),
               tcm.make_system(B, mB.center, mB.radius, moments=mB)]
    # the items are marshalled on the host before the timed GPU part (the library still packs
    # and uploads their descriptors inside the call)
    k = n * len(lmax_values)
    L_items = np.repeat(np.array(lmax_values), n)
    t0 = time.perf_counter()
    pb = tcm.pack_batch(systems, np.zeros(k, int), np.ones(k, int), L_items, np.tile(R0, (len(lmax_values), 1)))
    pack_ms = 1e3 * (time.perf_counter() - t0)
    ev[1].record(stream)
    E, st = ctx.tcm_energy_batch_packed(pb, precision)
    ev[2].record(stream)
    Ec = None
    if direct:
        Ec = ctx.tcm_direct_batch(A, B, R0, cA=mA.center, cB=mB.center)
    ev[3].record(stream)
    torch.cuda.synchronize()
    if not bool(torch.all(st == tcm.TCM_OK)):
        raise tcm.TcmError(tcm.TCM_ENOTCONV, "some grid points violate Eq. (mainCond)")
    Eh = E.cpu().numpy().reshape(len(lmax_values), n)
    res = PesResult(R0, lmax_values, {L: Eh[i] for i, L in enumerate(lmax_values)},
                    None if Ec is None else Ec.cpu().numpy())
    res.timings_ms = {"moments": ev[0].elapsed_time(ev[1]), "tcm_energies": ev[1].elapsed_time(ev[2]),
                      "item_packing_host": pack_ms,
                      "direct": ev[2].elapsed_time(ev[3]) if direct else None}
    res.centers = (mA.center, mB.center)
    res.radii = (mA.radius, mB.radius)
    return res


def main():
    """Command line: the Section IV surface scan on synthetic proteins; prints one JSON line with
    the timings, energies per second and the median and maximum of Eq. (error) per Lmax."""
    import argparse
    import json

    import torch

    from . import build, synth, tcm
    p = argparse.ArgumentParser(description="TCM surface scan (R0, Theta) with Eq. (error) maps")
    p.add_argument("--dr", type=float, default=1.0)
    p.add_argument("--dtheta", type=float, default=1.0)
    p.add_argument("--lmax", type=str, default="1,2,3,4,6,8,10")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--no-direct", action="store_true", help="skip the exact energies")
    p.add_argument("--repeat", type=int, default=2, help="scans run; the last is reported")
    args = p.parse_args()
    build.build()
    g = synth.pes_grid_pair(dr=args.dr, dtheta=args.dtheta, lmax=tuple(int(x) for x in args.lmax.split(",")))
    A = torch.tensor(g.A, device="cuda")
    B = torch.tensor(g.B, device="cuda")
    ctx = tcm.Context(lmax_cap=max(g.lmax))
    prec = tcm.TCM_MIXED if args.precision == "mixed" else tcm.TCM_FP64
    try:
        for _ in range(max(1, args.repeat)):
            res = scan(ctx, A, B, g.R0(), g.lmax, precision=prec, direct=not args.no_direct)
    finally:
        ctx.close()
    n = len(res.R0)
    out = {"workload": g.name, "points": n, "lmax": list(g.lmax), "timings_ms": res.timings_ms,
           "tcm_energies_per_s": n * len(g.lmax) / (res.timings_ms["tcm_energies"] * 1e-3)}
    if res.U_coul is not None:
        out["direct_pairs_per_s"] = n * len(g.A) * len(g.B) / (res.timings_ms["direct"] * 1e-3)
        out["eq_error_percent_median"] = {str(L): float(np.median(res.eta(L))) for L in g.lmax}
        out["eq_error_percent_max"] = {str(L): float(np.max(res.eta(L))) for L in g.lmax}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
