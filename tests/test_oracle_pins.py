"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test uses a closed form, an
exact rational, a library routine for a special function, brute-force Taylor
coefficients, an invariance or a bound, chosen so that a dropped term, a wrong
sign, index or conjugation, or a transposed operand in the oracle fails one of
them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_0704_1672_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def idx(l, m):
    return l * l + l + m


def rand_system(rng, n, radius, net_zero=True):
    pos = synth.uniform_ball(rng, n, radius)
    q = rng.uniform(-1, 1, n)
    if net_zero:
        q -= q.mean()
    return synth.pack(pos, q)


# ----------------------------------------------------------------------------- special functions

def test_threej_matches_exact_rationals():
    """Racah-sum 3j against sympy's exact values (all admissible args, j <= 4, plus stretched up to 12)."""
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import wigner_3j

    cases = []
    for j1 in range(5):
        for j2 in range(5):
            for j3 in range(abs(j1 - j2), j1 + j2 + 1):
                for m1 in range(-j1, j1 + 1):
                    for m2 in range(-j2, j2 + 1):
                        m3 = -m1 - m2
                        if abs(m3) <= j3:
                            cases.append((j1, j2, j3, m1, m2, m3))
    rng = np.random.default_rng(7)
    for _ in range(150):
        l1, l2 = rng.integers(0, 13, 2)
        m1 = int(rng.integers(-l1, l1 + 1))
        m2 = int(rng.integers(-l2, l2 + 1))
        cases.append((int(l1), int(l2), int(l1 + l2), m1, m2, -m1 - m2))
    worst = 0.0
    for c in cases:
        exact = float(wigner_3j(*c))
        got = oracle.threej(*c)
        worst = max(worst, abs(got - exact) / max(abs(exact), 1e-300) if exact != 0 else abs(got))
    assert worst < 1e-14
    # selection rule: m1 + m2 + m3 != 0 gives zero
    assert oracle.threej(2, 2, 2, 1, 1, 1) == 0.0


def test_ylm_matches_scipy_and_closed_forms():
    """Orthonormal Y_lm with Condon-Shortley phase: scipy's sph_harm_y and textbook low orders."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    for _ in range(40):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        for l in (0, 1, 2, 5, 13, 30, 48):
            for m in sorted({-l, -1 if l else 0, 0, 1 if l else 0, l // 2, l}):
                ref = complex(sp.sph_harm_y(l, m, th, ph))
                got = oracle.ylm(l, m, th, ph)
                assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (l, m)
    th, ph = 0.7, 1.1
    assert abs(oracle.ylm(1, 1, th, ph) - (-math.sqrt(3 / (8 * math.pi)) * math.sin(th) * complex(math.cos(ph), math.sin(ph)))) < 1e-15
    assert abs(oracle.ylm(1, 0, th, ph) - math.sqrt(3 / (4 * math.pi)) * math.cos(th)) < 1e-15
    assert abs(oracle.ylm(2, -2, th, ph) - math.sqrt(15 / (32 * math.pi)) * math.sin(th) ** 2 * complex(math.cos(2 * ph), -math.sin(2 * ph))) < 1e-15
    # near the poles (the oracle's series branch): closed forms, and scipy where both are accurate
    for th in (1e-9, 3e-3, math.pi - 3e-3, math.pi - 1e-9):
        st, ct = math.sin(th), math.cos(th)
        e = complex(math.cos(ph), math.sin(ph))
        assert abs(oracle.ylm(1, 1, th, ph) - (-math.sqrt(3 / (8 * math.pi)) * st * e)) < 1e-15 * max(st, 1e-300) + 1e-300
        assert abs(oracle.ylm(2, 1, th, ph) - (-math.sqrt(15 / (8 * math.pi)) * st * ct * e)) <= 1e-15 * st
        assert abs(oracle.ylm(3, 3, th, ph) - (-math.sqrt(35 / (64 * math.pi)) * st ** 3 * e ** 3)) <= 1e-14 * st ** 3
        assert abs(oracle.ylm(4, 0, th, ph) - 3 / (16 * math.sqrt(math.pi)) * (35 * ct ** 4 - 30 * ct ** 2 + 3)) < 1e-14
    for th in (0.012, 0.02, math.pi - 0.015):
        for l in (7, 24, 48):
            for m in (0, 1, 2, 5):
                ref = complex(sp.sph_harm_y(l, m, th, ph))
                assert abs(oracle.ylm(l, m, th, ph) - ref) <= 1e-12 * max(1.0, abs(ref)), (th, l, m)


# ----------------------------------------------------------------------------- moments, Eq. (multipole)

def test_moments_low_order_closed_forms():
    """Q_lm for l <= 2 written as Cartesian sums (Racah-normalised regular solid harmonics)."""
    rng = np.random.default_rng(11)
    S = rand_system(rng, 37, 3.0, net_zero=False)
    c = np.array([0.3, -0.2, 0.1])
    # atoms within 1e-9 of the poles: their polar angle must keep its digits
    S = np.vstack([S, [[c[0] + 1e-9, c[1] + 2e-9, c[2] + 1.3, 0.7], [c[0] - 3e-10, c[1] + 1e-10, c[2] - 0.7, -0.4]]])
    Q = oracle.moments(S, c, 3)
    x, y, z = (S[:, :3] - c).T
    q = S[:, 3]
    r2 = x * x + y * y + z * z
    w = x + 1j * y
    exp = {
        (0, 0): q.sum(),
        (1, 0): (q * z).sum(),
        (1, 1): -(q * w).sum() / math.sqrt(2),
        (1, -1): (q * np.conj(w)).sum() / math.sqrt(2),
        (2, 0): (q * (3 * z * z - r2) / 2).sum(),
        (2, 1): -math.sqrt(1.5) * (q * z * w).sum(),
        (2, -1): math.sqrt(1.5) * (q * z * np.conj(w)).sum(),
        (2, 2): math.sqrt(3 / 8) * (q * w * w).sum(),
        (2, -2): math.sqrt(3 / 8) * (q * np.conj(w) ** 2).sum(),
        (3, 3): -math.sqrt(5 / 16) * (q * w ** 3).sum(),
        (3, 0): (q * z * (5 * z * z - 3 * r2) / 2).sum(),
    }
    for (l, m), v in exp.items():
        assert abs(Q[idx(l, m)] - v) <= 1e-13 * max(1.0, abs(v)), (l, m)
    one = oracle.moments(np.array([[1e-9, 2e-9, 1.3, 1.0]]), np.zeros(3), 1)
    assert abs(one[idx(1, 1)] - (-(1e-9 + 2e-9j) / math.sqrt(2))) < 1e-24


def test_moments_addition_theorem_and_rotation():
    """One unit charge at distance r: sum_m |Q_lm|^2 = r^(2l); per-degree norms survive rotation."""
    rng = np.random.default_rng(5)
    L = 16
    for _ in range(5):
        p = rng.normal(size=3)
        r = np.linalg.norm(p)
        Q = oracle.moments(np.array([[*p, 1.0]]), np.zeros(3), L)
        for l in range(L + 1):
            s = np.sum(np.abs(Q[l * l:(l + 1) * (l + 1)]) ** 2)
            assert abs(s - r ** (2 * l)) <= 1e-12 * r ** (2 * l)
    S = rand_system(rng, 25, 2.0)
    R = synth.random_rotations(rng, 1)[0]
    Q0 = oracle.moments(S, np.zeros(3), L)
    Q1 = oracle.moments(S, np.zeros(3), L, rot=R)
    S_rot = S.copy()
    S_rot[:, :3] = S[:, :3] @ R.T
    Q2 = oracle.moments(S_rot, np.zeros(3), L)
    assert np.max(np.abs(Q1 - Q2)) < 1e-12 * np.max(np.abs(Q0))
    for l in range(L + 1):
        n0 = np.sum(np.abs(Q0[l * l:(l + 1) ** 2]) ** 2)
        n1 = np.sum(np.abs(Q1[l * l:(l + 1) ** 2]) ** 2)
        assert abs(n0 - n1) <= 1e-11 * n0
    # real charges: Q_l,-m = (-1)^m conj(Q_lm)
    for l in range(L + 1):
        for m in range(1, l + 1):
            assert abs(Q0[idx(l, -m)] - (-1) ** m * np.conj(Q0[idx(l, m)])) < 1e-13 * max(1, abs(Q0[idx(l, m)]))


def test_center_radius_by_hand():
    S = np.array([[1.0, 0, 0, 1], [-1.0, 0, 0, -1], [0, 3.0, 0, 2], [0, -3.0, 0, 0.5]])
    c, a = oracle.center_radius(S)
    assert np.allclose(c, 0.0, atol=0) and a == 3.0
    S2 = S.copy()
    S2[:, :3] += [10.0, -4.0, 2.5]
    c2, a2 = oracle.center_radius(S2)
    assert np.allclose(c2, [10.0, -4.0, 2.5], rtol=0, atol=1e-15) and abs(a2 - 3.0) < 1e-14


# ----------------------------------------------------------------------------- direct sum, Eq. (Coulomb)

def _read_direct_cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, "direct_hand_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *vals = line.split()
        vals = [float(v) for v in vals]
        if cur is None:
            cur = {"A": [], "B": []}
        if tag in ("A", "B"):
            cur[tag].append(vals)
        elif tag == "R0":
            cur["R0"] = np.array(vals)
        elif tag == "U":
            cur["U"] = vals[0]
            cases.append(cur)
            cur = None
    return cases


def test_direct_hand_cases():
    cases = _read_direct_cases()
    assert len(cases) == 4
    for c in cases:
        A, B = np.array(c["A"]), np.array(c["B"])
        U = oracle.direct(A, np.zeros(3), B, np.zeros(3), c["R0"])
        assert abs(U - c["U"]) < 1e-15 * max(1, abs(c["U"])) + 1e-16


def test_direct_rotation_and_symmetry():
    """Rotating B about its centre equals rotating its coordinates; swapping A and B with R0 -> -R0."""
    rng = np.random.default_rng(9)
    A = rand_system(rng, 30, 2.0)
    B = rand_system(rng, 20, 1.5)
    cA = np.array([1.0, 2.0, 3.0])
    A[:, :3] += cA
    cB = np.array([-2.0, 0.5, 0.0])
    B[:, :3] += cB
    R0 = np.array([3.0, -4.0, 6.0])
    Rot = synth.random_rotations(rng, 1)[0]
    U1 = oracle.direct(A, cA, B, cB, R0, rotB=Rot)
    B2 = B.copy()
    B2[:, :3] = (B[:, :3] - cB) @ Rot.T + cB
    U2 = oracle.direct(A, cA, B2, cB, R0)
    assert abs(U1 - U2) < 1e-13
    U3 = oracle.direct(B2, cB, A, cA, -R0)
    assert abs(U2 - U3) < 1e-13


# ----------------------------------------------------------------------------- energy, Eq. (Formula)

def test_energy_monopole_is_qaqb_over_r():
    rng = np.random.default_rng(1)
    A = rand_system(rng, 12, 1.0, net_zero=False)
    B = rand_system(rng, 9, 1.0, net_zero=False)
    R0 = np.array([2.0, -5.0, 3.0])
    U = oracle.tcm_energy_systems(A, B, 0, R0, cA=np.zeros(3), cB=np.zeros(3))
    assert abs(U - A[:, 3].sum() * B[:, 3].sum() / np.linalg.norm(R0)) < 1e-14


def test_energy_lmax1_charge_dipole_and_dipole_dipole():
    """Lmax = 1: monopole + charge-dipole + dipole-dipole closed forms (Taylor expansion of Eq. (Coulomb))."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        A = rand_system(rng, 15, 1.0, net_zero=False)
        B = rand_system(rng, 11, 1.3, net_zero=False)
        R0 = synth.unit_vectors(rng, 1)[0] * rng.uniform(5, 9)
        Rn = np.linalg.norm(R0)
        Rh = R0 / Rn
        qa, qb = A[:, 3].sum(), B[:, 3].sum()
        pa = (A[:, 3:4] * A[:, :3]).sum(0)
        pb = (B[:, 3:4] * B[:, :3]).sum(0)
        exp = qa * qb / Rn + (qb * pa @ R0 - qa * pb @ R0) / Rn ** 3 + (pa @ pb - 3 * (pa @ Rh) * (pb @ Rh)) / Rn ** 3
        U, im = oracle.tcm_energy(1, oracle.moments(A, np.zeros(3), 1), oracle.moments(B, np.zeros(3), 1), R0, return_imag=True)
        assert abs(U - exp) < 1e-14 * max(1, abs(exp))
        assert abs(im) < 1e-15


def _collinear_blocks(L, sa, sb, R):
    """Charge +1 at sa*Rhat in A and +1 at sb*Rhat in B: 1/(R + sb - sa) expanded in sa and sb."""
    out = np.zeros((L + 1, L + 1))
    for l1 in range(L + 1):
        for l2 in range(L + 1):
            out[l1, l2] = math.comb(l1 + l2, l1) * sa ** l1 * (-sb) ** l2 / R ** (l1 + l2 + 1)
    return out


def test_energy_collinear_every_block_and_golden_values():
    """Every (l1, l2) block in the collinear geometry, along random directions, L up to 12."""
    rng = np.random.default_rng(4)
    for _ in range(6):
        Rh = synth.unit_vectors(rng, 1)[0]
        R = rng.uniform(6, 10)
        sa, sb = rng.uniform(-2, 2), rng.uniform(-2, 2)
        L = 12
        QA = oracle.moments(np.array([[*(sa * Rh), 1.0]]), np.zeros(3), L)
        QB = oracle.moments(np.array([[*(sb * Rh), 1.0]]), np.zeros(3), L)
        blk = oracle.tcm_blocks(L, QA, QB, R * Rh)
        exp = _collinear_blocks(L, sa, sb, R)
        assert np.max(np.abs(blk.real - exp)) < 1e-13 * np.max(np.abs(exp))
        assert np.max(np.abs(blk.imag)) < 1e-14 * np.max(np.abs(exp))
    # the printed example (a = 1, b = 1.5, R = 5): partial sums rise monotonically to 0.4
    rows = [l.split() for l in open(os.path.join(GOLDEN, "collinear_a1_b1.5_R5.txt")) if l.strip() and not l.startswith("#")]
    Rh = np.array([0.0, 0.0, 1.0])
    prev = -1.0
    for lm, val in rows:
        if lm == "inf":
            assert prev < float(val)
            continue
        L = int(lm)
        QA = oracle.moments(np.array([[0, 0, 1.0, 1.0]]), np.zeros(3), L)
        QB = oracle.moments(np.array([[0, 0, -1.5, 1.0]]), np.zeros(3), L)
        U = oracle.tcm_energy(L, QA, QB, 5.0 * Rh)
        assert abs(U - float(val)) < 1e-15
        assert U > prev
        prev = U


def _taylor_blocks(A, B, R0, L, K=64):
    """Brute force: block (l1, l2) = coefficient of s^l1 t^l2 of
    f(s, t) = sum_ij q_i q_j / sqrt(|R0 + t r_j - s r_i|^2) (principal branch),
    extracted by a 2-D FFT on the circles |s| = |t| = rho."""
    ra, qa = A[:, :3], A[:, 3]
    rb, qb = B[:, :3], B[:, 3]
    R = np.linalg.norm(R0)
    amax = np.linalg.norm(ra, axis=1).max()
    bmax = np.linalg.norm(rb, axis=1).max()
    rho = 0.35 * R / (amax + bmax)
    w = rho * np.exp(2j * np.pi * np.arange(K) / K)
    s = w[:, None, None, None]
    t = w[None, :, None, None]
    d = R0[None, None, None, None, :] + t[..., None] * rb[None, None, None, :, :] - s[..., None] * ra[None, None, :, None, :]
    D = np.sum(d * d, axis=-1)
    f = np.sum(qa[None, None, :, None] * qb[None, None, None, :] / np.sqrt(D), axis=(2, 3))
    c = np.fft.fft2(f) / K ** 2
    out = np.zeros((L + 1, L + 1), dtype=complex)
    for l1 in range(L + 1):
        for l2 in range(L + 1):
            out[l1, l2] = c[l1, l2] / rho ** (l1 + l2)
    return out


def test_energy_blocks_match_brute_force_taylor_coefficients():
    """General geometry, every (l1, l2) block up to Lmax = 6 against an FFT Taylor extraction."""
    rng = np.random.default_rng(6)
    for _ in range(3):
        A = rand_system(rng, 4, 1.0)
        B = rand_system(rng, 3, 1.2)
        R0 = synth.unit_vectors(rng, 1)[0] * 4.0
        L = 6
        blk = oracle.tcm_blocks(L, oracle.moments(A, np.zeros(3), L), oracle.moments(B, np.zeros(3), L), R0)
        ref = _taylor_blocks(A, B, R0, L)
        scale = np.abs(ref).max()
        assert np.max(np.abs(blk.real - ref.real)) < 1e-9 * scale
        assert np.max(np.abs(blk.imag)) < 1e-14 * scale


def test_single_pair_converges_to_coulomb():
    """One charge per system: U_L -> q1 q2 / |R0 + r2 - r1| geometrically (Eq. (SpherHarm_exp2))."""
    rng = np.random.default_rng(8)
    r1 = synth.unit_vectors(rng, 1)[0] * 1.0
    r2 = synth.unit_vectors(rng, 1)[0] * 0.8
    R0 = synth.unit_vectors(rng, 1)[0] * 4.5
    A = np.array([[*r1, 0.7]])
    B = np.array([[*r2, -1.3]])
    exact = oracle.direct(A, np.zeros(3), B, np.zeros(3), R0)
    errs = []
    for L in range(0, 25, 4):
        U = oracle.tcm_energy_systems(A, B, L, R0, cA=np.zeros(3), cB=np.zeros(3))
        errs.append(abs(U - exact))
    assert errs[-1] < 1e-10 * abs(exact)
    assert errs[-1] < errs[0] * 1e-6


def _bound(A, B, R, L):
    """sum_ij |q_i q_j| [1/(R - r_i - r_j) - S_L(r_i, r_j)], S_L the collinear partial sum."""
    ra = np.linalg.norm(A[:, :3], axis=1)
    rb = np.linalg.norm(B[:, :3], axis=1)
    total = 0.0
    for i in range(len(A)):
        for j in range(len(B)):
            S = sum(math.comb(l1 + l2, l1) * ra[i] ** l1 * rb[j] ** l2 / R ** (l1 + l2 + 1)
                    for l1 in range(L + 1) for l2 in range(L + 1))
            total += abs(A[i, 3] * B[j, 3]) * (1.0 / (R - ra[i] - rb[j]) - S)
    return total


def test_truncation_error_within_monotone_bound():
    """Under Eq. (mainCond), |U_Coulomb - U_L| stays below a bound that falls monotonically with L."""
    rng = np.random.default_rng(10)
    for _ in range(4):
        A = rand_system(rng, 6, 1.0)
        B = rand_system(rng, 5, 1.0)
        aA = np.linalg.norm(A[:, :3], axis=1).max()
        aB = np.linalg.norm(B[:, :3], axis=1).max()
        R0 = synth.unit_vectors(rng, 1)[0] * 1.25 * (aA + aB)
        R = np.linalg.norm(R0)
        exact = oracle.direct(A, np.zeros(3), B, np.zeros(3), R0)
        QA = oracle.moments(A, np.zeros(3), 14)
        QB = oracle.moments(B, np.zeros(3), 14)
        prev = math.inf
        for L in range(0, 15):
            err = abs(oracle.tcm_energy(L, QA, QB, R0) - exact)
            b = _bound(A, B, R, L)
            assert err <= b * (1 + 1e-9) + 1e-15
            assert b < prev
            prev = b


def test_energy_invariances():
    """Joint rotation of A, B and R0; swapping A and B with R0 -> -R0; linearity in the charges."""
    rng = np.random.default_rng(12)
    A = rand_system(rng, 10, 1.0)
    B = rand_system(rng, 8, 1.0)
    R0 = synth.unit_vectors(rng, 1)[0] * 5.0
    L = 10
    z = np.zeros(3)
    U = oracle.tcm_energy_systems(A, B, L, R0, cA=z, cB=z)
    Rot = synth.random_rotations(rng, 1)[0]
    Ar, Br = A.copy(), B.copy()
    Ar[:, :3] = A[:, :3] @ Rot.T
    Br[:, :3] = B[:, :3] @ Rot.T
    assert abs(oracle.tcm_energy_systems(Ar, Br, L, Rot @ R0, cA=z, cB=z) - U) < 1e-13 * abs(U) + 1e-17
    assert abs(oracle.tcm_energy_systems(B, A, L, -R0, cA=z, cB=z) - U) < 1e-13 * abs(U) + 1e-17
    A2 = A.copy()
    A2[:, 3] *= -2.5
    assert abs(oracle.tcm_energy_systems(A2, B, L, R0, cA=z, cB=z) + 2.5 * U) < 1e-13 * abs(U) + 1e-17
    # rotating B about its centre inside the oracle equals rotating B's coordinates
    assert abs(oracle.tcm_energy_systems(A, B, L, R0, rotB=Rot, cA=z, cB=z)
               - oracle.tcm_energy_systems(A, Br, L, R0, cA=z, cB=z)) < 1e-13 * abs(U) + 1e-17
