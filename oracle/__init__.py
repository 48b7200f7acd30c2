"""Plain CPU oracle for the two-center multipole method (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and the
CUDA path shares no code with it.

Functions follow the paper's equations (cited per function in
``tcm_oracle.cpp``): Eq. (Coulomb) for the exact energy, Eq. (multipole) for the
moments, Eq. (3j) / Racah for the coupling, Eq. (Formula) for the truncated
two-center energy; the gradient of Eq. (Formula) in R0, the derivative of Eq. (multipole)
under a rotation, and the exact pairwise forces and torques for the forces and torques.
Moments are complex arrays of length (L+1)^2 indexed
``l*l + l + m`` for ``m = -l..l``.

Parity status: every function here is pinned in ``tests/test_oracle_pins.py``
(closed forms, brute-force Taylor coefficients, library routines, invariants).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        lib.oracle_abi_version.restype = i32
        lib.oracle_center_radius.argtypes = [i64, P, P, P]
        lib.oracle_ylm.argtypes = [i32, i32, d, d, P, P]
        lib.oracle_threej.argtypes = [i32] * 6
        lib.oracle_threej.restype = d
        lib.oracle_moments.argtypes = [i64, P, P, P, i32, P, P]
        lib.oracle_tcm_blocks.argtypes = [i32, P, P, P, P, P, P, P]
        lib.oracle_tcm_energy.argtypes = [i32, P, P, P, P, P, P]
        lib.oracle_tcm_energy.restype = d
        lib.oracle_direct.argtypes = [i64, P, P, i64, P, P, P, P, P]
        lib.oracle_direct.restype = d
        lib.oracle_tcm_force.argtypes = [i32, P, P, P, P, P, P, P]
        lib.oracle_moments_rotderiv.argtypes = [i64, P, P, P, i32, P, P, P]
        lib.oracle_direct_forces.argtypes = [i64, P, P, i64, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def center_radius(xyzq):
    """Centroid (unit masses) and radius a = max |x_i - c| of one system."""
    xyzq = _f64(xyzq, (-1, 4))
    c = np.zeros(3)
    a = np.zeros(1)
    _load().oracle_center_radius(xyzq.shape[0], _ptr(xyzq), _ptr(c), _ptr(a))
    return c, float(a[0])


def ylm(l, m, theta, phi):
    """Orthonormal Y_lm(theta, phi), Condon-Shortley phase."""
    re = np.zeros(1)
    im = np.zeros(1)
    _load().oracle_ylm(l, m, float(theta), float(phi), _ptr(re), _ptr(im))
    return complex(re[0], im[0])


def threej(j1, j2, j3, m1, m2, m3):
    """Wigner 3j symbol (Racah sum)."""
    return _load().oracle_threej(j1, j2, j3, m1, m2, m3)


def moments(xyzq, center, L, rot=None):
    """Eq. (multipole): complex Q_lm, index l*l+l+m, about ``center`` (rotated by ``rot``)."""
    xyzq = _f64(xyzq, (-1, 4))
    c = _f64(center, (3,))
    r = None if rot is None else _f64(rot, (9,))
    n = (L + 1) ** 2
    re = np.zeros(n)
    im = np.zeros(n)
    _load().oracle_moments(xyzq.shape[0], _ptr(xyzq), _ptr(c), _ptr(r), int(L), _ptr(re), _ptr(im))
    return re + 1j * im


def tcm_blocks(L, QA, QB, R0):
    """Eq. (Formula) resolved per (l1, l2): returns an (L+1, L+1) complex array."""
    QA = np.asarray(QA, dtype=np.complex128)
    QB = np.asarray(QB, dtype=np.complex128)
    n = (L + 1) ** 2
    QA, QB = QA[:n], QB[:n]
    ar, ai = _f64(QA.real), _f64(QA.imag)
    br, bi = _f64(QB.real), _f64(QB.imag)
    R = _f64(R0, (3,))
    out = np.zeros((L + 1) * (L + 1))
    out_i = np.zeros((L + 1) * (L + 1))
    _load().oracle_tcm_blocks(int(L), _ptr(ar), _ptr(ai), _ptr(br), _ptr(bi), _ptr(R), _ptr(out), _ptr(out_i))
    return (out + 1j * out_i).reshape(L + 1, L + 1)


def tcm_energy(L, QA, QB, R0, return_imag=False):
    """Eq. (Formula): U_mult truncated at Lmax = L (square truncation l1, l2 <= L).

    ``QA`` and ``QB`` may carry more than (L+1)^2 components; the leading ones are used.
    """
    QA = np.asarray(QA, dtype=np.complex128)
    QB = np.asarray(QB, dtype=np.complex128)
    n = (L + 1) ** 2
    QA, QB = QA[:n], QB[:n]
    ar, ai = _f64(QA.real), _f64(QA.imag)
    br, bi = _f64(QB.real), _f64(QB.imag)
    R = _f64(R0, (3,))
    im = np.zeros(1)
    e = _load().oracle_tcm_energy(int(L), _ptr(ar), _ptr(ai), _ptr(br), _ptr(bi), _ptr(R), _ptr(im))
    return (e, float(im[0])) if return_imag else e


def direct(A, cA, B, cB, R0, rotB=None, return_abs=False):
    """Eq. (Coulomb): exact pairwise energy with B rotated about its centre by ``rotB``.

    With ``return_abs`` also returns sum_ij |q_i q_j| / r_ij (the rounding scale of the sum).
    """
    A = _f64(A, (-1, 4))
    B = _f64(B, (-1, 4))
    ca = _f64(cA, (3,))
    cb = _f64(cB, (3,))
    r = None if rotB is None else _f64(rotB, (9,))
    R = _f64(R0, (3,))
    ab = np.zeros(1)
    e = _load().oracle_direct(A.shape[0], _ptr(A), _ptr(ca), B.shape[0], _ptr(B), _ptr(cb), _ptr(r), _ptr(R), _ptr(ab))
    return (e, float(ab[0])) if return_abs else e


def tcm_energy_systems(A, B, L, R0, rotB=None, cA=None, cB=None):
    """Convenience: centres (centroids unless given), moments and Eq. (Formula) energy."""
    if cA is None:
        cA, _ = center_radius(A)
    if cB is None:
        cB, _ = center_radius(B)
    QA = moments(A, cA, L)
    QB = moments(B, cB, L, rot=rotB)
    return tcm_energy(L, QA, QB, R0)


def tcm_force(L, QA, QB, R0, return_blocks=False):
    """Force on B, -grad_R0 of Eq. (Formula) (the separation harmonic differentiated with the
    textbook derivatives of Y_LM).  With ``return_blocks`` also the per-(l1, l2) block force
    lengths, shape (L+1, L+1)."""
    QA = np.asarray(QA, dtype=np.complex128)[:(L + 1) ** 2]
    QB = np.asarray(QB, dtype=np.complex128)[:(L + 1) ** 2]
    ar, ai = _f64(QA.real), _f64(QA.imag)
    br, bi = _f64(QB.real), _f64(QB.imag)
    R = _f64(R0, (3,))
    F = np.zeros(3)
    bn = np.zeros((L + 1) * (L + 1))
    _load().oracle_tcm_force(int(L), _ptr(ar), _ptr(ai), _ptr(br), _ptr(bi), _ptr(R), _ptr(F), _ptr(bn))
    return (F, bn.reshape(L + 1, L + 1)) if return_blocks else F


def moments_rotderiv(xyzq, center, L, axis, rot=None):
    """d/d(eps) of Eq. (multipole) when the system (after ``rot``) turns by eps about ``axis``
    through its centre: complex array indexed l*l + l + m."""
    x = _f64(xyzq, (-1, 4))
    c = _f64(center, (3,))
    r = None if rot is None else _f64(rot, (9,))
    ax = _f64(axis, (3,))
    n = (L + 1) * (L + 1)
    dr, di = np.zeros(n), np.zeros(n)
    _load().oracle_moments_rotderiv(x.shape[0], _ptr(x), _ptr(c), _ptr(r), int(L), _ptr(ax), _ptr(dr), _ptr(di))
    return dr + 1j * di


def tcm_torques(L, QA, QB, R0, dQA, dQB):
    """Torques on A and on B about their centres from Eq. (Formula), which is linear in each
    moment set: tau_X . n = -U_mult(with Q_X replaced by dQ_X/d(eps) about n).  ``dQA``/``dQB``
    are the three derivatives (``moments_rotderiv`` about x, y, z)."""
    tA = np.array([-tcm_energy(L, dQA[k], QB, R0) for k in range(3)])
    tB = np.array([-tcm_energy(L, QA, dQB[k], R0) for k in range(3)])
    return tA, tB


def tcm_gradients_systems(A, cA, B, cB, L, R0, rotB=None):
    """Energy, force on B and torques on A and B of Eq. (Formula) for two systems."""
    QA = moments(A, cA, L)
    QB = moments(B, cB, L, rot=rotB)
    eye = np.eye(3)
    dQA = [moments_rotderiv(A, cA, L, eye[k]) for k in range(3)]
    dQB = [moments_rotderiv(B, cB, L, eye[k], rot=rotB) for k in range(3)]
    tA, tB = tcm_torques(L, QA, QB, R0, dQA, dQB)
    return tcm_energy(L, QA, QB, R0), tcm_force(L, QA, QB, R0), tA, tB


def direct_forces(A, cA, B, cB, R0, rotB=None):
    """Exact pairwise force on B and torques on A and B (Eq. (Coulomb) differentiated), and
    the scale sum_ij |q_i q_j| / r_ij^2.  Returns (F_B, tau_A, tau_B, scale)."""
    A = _f64(A, (-1, 4))
    B = _f64(B, (-1, 4))
    ca = _f64(cA, (3,))
    cb = _f64(cB, (3,))
    r = None if rotB is None else _f64(rotB, (9,))
    R = _f64(R0, (3,))
    out = np.zeros(9)
    ab = np.zeros(1)
    _load().oracle_direct_forces(A.shape[0], _ptr(A), _ptr(ca), B.shape[0], _ptr(B), _ptr(cb), _ptr(r), _ptr(R),
                                 _ptr(out), _ptr(ab))
    return out[:3], out[3:6], out[6:], float(ab[0])
