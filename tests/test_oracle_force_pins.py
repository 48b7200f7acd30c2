"""Pins of the oracle's forces and torques (CPU, no GPU).

The paper names forces as a use of Eq. (Formula) but prints no formula, so the oracle
differentiates its own definitions; these tests tie that to things fixed independently:
finite differences of the oracle energies, the collinear closed form, the low-order closed
forms, Newton's third law for torques (angular-momentum balance, exact for the square
truncation because every (l1, l2) block is rotation invariant), and convergence to the exact
pairwise forces and torques of Eq. (Coulomb), themselves pinned by finite differences."""
import numpy as np
import pytest
from math import comb

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def ball_system(seed, n, r):
    g = np.random.default_rng(seed)
    x = g.normal(size=(n, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    x *= r * g.random((n, 1)) ** (1 / 3)
    q = g.uniform(-1, 1, n)
    q -= q.mean()
    return np.c_[x, q]


def rod(axis, ang):
    k = np.asarray(axis, dtype=float)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


DIRECTIONS = [np.array([3.0, -4.0, 5.5]), np.array([1e-4, 2e-4, 7.0]), np.array([0.3, -0.2, -6.5]),
              np.array([-5.0, 2.0, 0.0])]


@pytest.mark.parametrize("k", range(len(DIRECTIONS)))
def test_force_is_minus_gradient_of_energy(k):
    A, B = ball_system(1, 8, 2.0), ball_system(2, 7, 1.5)
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    L = 7
    QA, QB = oracle.moments(A, cA, L), oracle.moments(B, cB, L, rot=rod([1, 1, 0], 0.4))
    R0 = DIRECTIONS[k]
    F, blocks = oracle.tcm_force(L, QA, QB, R0, return_blocks=True)
    G = np.array([richardson(lambda t: oracle.tcm_energy(L, QA, QB, R0 + t * e), 1e-3) for e in np.eye(3)])
    assert np.linalg.norm(F + G) < 1e-8 * blocks.sum(), (F, -G)


def test_force_collinear_closed_form():
    """Unit charges at a Rhat in A and -b Rhat in B: F_B = Rhat sum C(l1+l2, l1) a^l1 b^l2 (L+1)/R^(L+2)."""
    rng = np.random.default_rng(3)
    a, b, R, L = 1.0, 1.5, 5.0, 12
    for _ in range(4):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        A = np.array([[*(a * u), 1.0]])
        B = np.array([[*(-b * u), 1.0]])
        c0 = np.zeros(3)
        QA, QB = oracle.moments(A, c0, L), oracle.moments(B, c0, L)
        F = oracle.tcm_force(L, QA, QB, R * u)
        mag = sum(comb(l1 + l2, l1) * a ** l1 * b ** l2 * (l1 + l2 + 1) / R ** (l1 + l2 + 2)
                  for l1 in range(L + 1) for l2 in range(L + 1))
        assert np.allclose(F, mag * u, rtol=0, atol=1e-13 * mag)


def test_force_through_dipole_order_closed_form():
    A, B = ball_system(5, 6, 1.0), ball_system(6, 5, 1.2)
    A[:, 3] += 0.3  # net charges too
    B[:, 3] -= 0.2
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    QAt, QBt = A[:, 3].sum(), B[:, 3].sum()
    pA = (A[:, 3:4] * (A[:, :3] - cA)).sum(0)
    pB = (B[:, 3:4] * (B[:, :3] - cB)).sum(0)
    R0 = np.array([2.0, 3.5, -4.0])
    R = np.linalg.norm(R0)
    grad = (-QAt * QBt * R0 / R ** 3
            + QBt * (pA / R ** 3 - 3 * (pA @ R0) * R0 / R ** 5)
            - QAt * (pB / R ** 3 - 3 * (pB @ R0) * R0 / R ** 5)
            - 3 * (pA @ pB) * R0 / R ** 5
            - 3 * ((pA * (pB @ R0) + pB * (pA @ R0)) / R ** 5 - 5 * (pA @ R0) * (pB @ R0) * R0 / R ** 7))
    F = oracle.tcm_force(1, oracle.moments(A, cA, 1), oracle.moments(B, cB, 1), R0)
    assert np.allclose(F, -grad, rtol=0, atol=1e-14 * np.abs(grad).max())
    F0 = oracle.tcm_force(0, oracle.moments(A, cA, 0), oracle.moments(B, cB, 0), R0)
    assert np.allclose(F0, QAt * QBt * R0 / R ** 3, rtol=1e-14, atol=0)


def test_monopole_force_direction_near_the_pole():
    A = np.array([[0.0, 0.0, 0.0, 0.8]])
    B = np.array([[0.0, 0.0, 0.0, -0.6]])
    for R0 in (np.array([1e-9, 0.0, 25.0]), np.array([0.0, -2e-10, -25.0])):
        F = oracle.tcm_force(0, oracle.moments(A, np.zeros(3), 0), oracle.moments(B, np.zeros(3), 0), R0)
        R = np.linalg.norm(R0)
        assert np.allclose(F, 0.8 * -0.6 * R0 / R ** 3, rtol=0, atol=1e-15 * 0.48 / R ** 2)


def test_rotation_derivative_of_moments_matches_finite_differences():
    B = ball_system(7, 9, 1.5)
    B = np.vstack([B, [[1e-3, 2e-3, 1.0, 0.4], [0.0, 0.0, -0.8, -0.4]]])  # atoms at the poles
    cB = np.zeros(3)
    L = 8
    rot = rod([1, 2, 3], 0.7)
    for ax in list(np.eye(3)) + [np.array([0.6, 0.0, 0.8])]:
        d = oracle.moments_rotderiv(B, cB, L, ax, rot=rot)
        h = 1e-5
        fd = (oracle.moments(B, cB, L, rot=rod(ax, h) @ rot) - oracle.moments(B, cB, L, rot=rod(ax, -h) @ rot)) / (2 * h)
        assert np.max(np.abs(d - fd)) < 1e-8 * np.max(np.abs(d)), ax
        # an axis is a vector: the derivative is linear in it
    d3 = [oracle.moments_rotderiv(B, cB, L, e, rot=rot) for e in np.eye(3)]
    n = np.array([0.6, 0.0, 0.8])
    assert np.allclose(oracle.moments_rotderiv(B, cB, L, n, rot=rot), sum(n[k] * d3[k] for k in range(3)),
                       rtol=0, atol=1e-13 * np.max(np.abs(d3)))


@pytest.mark.parametrize("L", [0, 1, 3, 9])
def test_torques_balance_force_moment(L):
    """tau_A + tau_B + R0 x F_B = 0 for the truncated energy (each block is rotation invariant)."""
    A, B = ball_system(8, 8, 2.0), ball_system(9, 6, 1.2)
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    R0 = np.array([-3.0, 4.5, 2.0])
    E, F, tA, tB = oracle.tcm_gradients_systems(A, cA, B, cB, L, R0, rotB=rod([0, 1, 1], 1.1))
    scale = np.linalg.norm(tA) + np.linalg.norm(tB) + np.linalg.norm(np.cross(R0, F)) + 1e-30
    assert np.linalg.norm(tA + tB + np.cross(R0, F)) < 1e-12 * scale
    if L == 0:
        assert np.allclose(tA, 0, atol=1e-18) and np.allclose(tB, 0, atol=1e-18)


def test_direct_forces_match_finite_differences():
    A, B = ball_system(10, 7, 1.5), ball_system(11, 6, 1.0)
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    R0 = np.array([1.0, -2.0, 3.5])
    rot = rod([2, -1, 1], 0.9)
    F, tA, tB, sc = oracle.direct_forces(A, cA, B, cB, R0, rotB=rot)
    G = np.array([richardson(lambda t: oracle.direct(A, cA, B, cB, R0 + t * e, rotB=rot), 1e-3) for e in np.eye(3)])
    assert np.linalg.norm(F + G) < 1e-9 * sc
    dB = np.array([richardson(lambda t: oracle.direct(A, cA, B, cB, R0, rotB=rod(e, t) @ rot), 1e-3)
                   for e in np.eye(3)])
    assert np.linalg.norm(tB + dB) < 1e-9 * sc

    def rotated_A(e, t):
        Ar = A.copy()
        Ar[:, :3] = (A[:, :3] - cA) @ rod(e, t).T + cA
        return Ar
    dA = np.array([richardson(lambda t: oracle.direct(rotated_A(e, t), cA, B, cB, R0, rotB=rot), 1e-3)
                   for e in np.eye(3)])
    assert np.linalg.norm(tA + dA) < 1e-9 * sc
    assert np.linalg.norm(tA + tB + np.cross(R0, F)) < 1e-13 * sc * np.linalg.norm(R0)


def test_tcm_forces_and_torques_converge_to_exact():
    A, B = ball_system(12, 10, 2.0), ball_system(13, 8, 1.5)
    cA, aA = oracle.center_radius(A)
    cB, aB = oracle.center_radius(B)
    u = np.array([0.48, -0.6, 0.64])
    R0 = 2.5 * (aA + aB) * u / np.linalg.norm(u)
    rot = rod([1, 0, 2], 0.3)
    Fd, tAd, tBd, sc = oracle.direct_forces(A, cA, B, cB, R0, rotB=rot)
    errs = []
    for L in (4, 8, 12, 16, 20):
        _, F, tA, tB = oracle.tcm_gradients_systems(A, cA, B, cB, L, R0, rotB=rot)
        errs.append(max(np.linalg.norm(F - Fd), np.linalg.norm(tA - tAd), np.linalg.norm(tB - tBd)) / sc)
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-8, errs
