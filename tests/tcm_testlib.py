"""Shared helpers for the parity tests: tolerance measures and threaded oracle calls.

Tolerances (readings of the paper recorded in the design doc):
  * moments, per degree l:  max_m |dQ_lm| / max(||Q_l.||_2, KAPPA * S_l)
        where S_l = sum_i |q_i| r_i^l is the magnitude scale of the degree-l sum; a
        degree whose norm cancels below KAPPA * S_l is measured against that floor.
  * energy, double path: |dE| / max(|E|, 1e-3 * sum_{l1,l2} |U_l1l2|)
  * energy, mixed path: |dE| / sum_{l1,l2} |U_l1l2|  (the condition scale of Eq. (Formula); equal
        to |E| when the (l1, l2) blocks do not cancel).  Float per-atom arithmetic leaves each
        moment term with a relative error of about l * 2^-24 that no reduction removes, so the
        mixed path's energy error is bounded by the magnitudes of the blocks, not by |E|.
  * direct sum: |dU| / sum_ij |q_i q_j| / r_ij
  * bars: 1e-12 for the double path, 1e-5 (moments) and 1e-6 (energy) for the mixed path.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np

import oracle

KAPPA = 1e-3
TOL_FP64 = 1e-12
TOL_MIX_MOM = 1e-5
TOL_MIX_E = 1e-6


def degree_scales(xyzq, center, L, rot=None):
    d = xyzq[:, :3] - center
    if rot is not None:
        d = d @ np.asarray(rot).T
    r = np.sqrt((d * d).sum(1))
    q = np.abs(xyzq[:, 3])
    return np.array([(q * r ** l).sum() for l in range(L + 1)])


def moment_error(Q_test, Q_ref, S):
    """Per-degree error of complex moment arrays (index l*l+l+m); returns the max over degrees."""
    L = len(S) - 1
    worst = 0.0
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        den = max(np.linalg.norm(Q_ref[sl]), KAPPA * S[l])
        if den == 0.0:
            err = np.max(np.abs(Q_test[sl]))
        else:
            err = np.max(np.abs(Q_test[sl] - Q_ref[sl])) / den
        worst = max(worst, err)
    return worst


def energy_error(E_test, E_ref, blocks, mixed=False):
    if mixed:
        scale = np.sum(np.abs(blocks))
    else:
        scale = max(abs(E_ref), 1e-3 * np.sum(np.abs(blocks)))
    return abs(E_test - E_ref) / scale


def energy_error_vs_e(E_test, E_ref):
    return abs(E_test - E_ref) / abs(E_ref)


_POOL = None


def pool():
    global _POOL
    if _POOL is None:
        _POOL = ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2))
    return _POOL


def oracle_moments_threaded(xyzq, center, L, rot=None, parts=None):
    """Oracle Eq. (multipole) split over atom ranges in host threads (ctypes releases the GIL);
    the partial moment sums are added in a fixed order."""
    n = len(xyzq)
    parts = parts or min(max(1, n // 2000), 4 * (os.cpu_count() or 2))
    if parts <= 1:
        return oracle.moments(xyzq, center, L, rot=rot)
    bounds = np.linspace(0, n, parts + 1).astype(int)
    futs = [pool().submit(oracle.moments, xyzq[bounds[k]:bounds[k + 1]], center, L, rot) for k in range(parts)]
    out = np.zeros((L + 1) ** 2, dtype=np.complex128)
    for f in futs:
        out += f.result()
    return out


def oracle_direct_threaded(A, cA, B, cB, R0, rotB=None, parts=None):
    n = len(A)
    parts = parts or min(max(1, n // 500), 4 * (os.cpu_count() or 2))
    bounds = np.linspace(0, n, parts + 1).astype(int)
    futs = [pool().submit(oracle.direct, A[bounds[k]:bounds[k + 1]], cA, B, cB, R0, rotB, True) for k in range(parts)]
    e = s = 0.0
    for f in futs:
        a, b = f.result()
        e += a
        s += b
    return e, s
