"""Forces and torques (tcm_gradients_batch) against the oracle's derivatives of Eq. (Formula):
the force on B is -grad_R0 of the truncated energy, the torques are minus its derivatives under
rotations of A and of B about their centres.

Error measures: force |dF| / max(|F|, 1e-3 S_F), with S_F the sum of the (l1, l2) block force
lengths; torques the same against |R0| S_F.  The mixed path's bar is applied as for energies
(tcm_testlib.MixedEnergyReport)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import TOL_FP64, MixedEnergyReport, oracle_moments_threaded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tcm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0704_1672_gb300 import build
    build.build()
    from paper_0704_1672_gb300 import tcm as t
    torch.cuda.set_device(0)
    return t


@pytest.fixture(scope="module")
def ctx(tcm):
    c = tcm.Context(lmax_cap=24)
    yield c
    c.close()


def oracle_grads(A, cA, B, cB, L, R0, rot):
    QA = oracle_moments_threaded(A, cA, L)
    QB = oracle_moments_threaded(B, cB, L, rot=rot)
    eye = np.eye(3)
    dQA = [oracle.moments_rotderiv(A, cA, L, eye[k]) for k in range(3)]
    dQB = [oracle.moments_rotderiv(B, cB, L, eye[k], rot=rot) for k in range(3)]
    tA, tB = oracle.tcm_torques(L, QA, QB, R0, dQA, dQB)
    F, blocks = oracle.tcm_force(L, QA, QB, R0, return_blocks=True)
    return oracle.tcm_energy(L, QA, QB, R0), F, tA, tB, blocks.sum()


def errors(G, F, tA, tB, SF, R0, mixed=False):
    R = np.linalg.norm(R0)
    def err(v, ref, S):
        return np.linalg.norm(v - ref) / max(np.linalg.norm(ref), 1e-3 * S)
    return err(G[:3], F, SF), err(G[3:6], tA, R * SF), err(G[6:], tB, R * SF)


def test_single_pair_fp64_forces_and_torques(ctx, tcm):
    s = synth.single_pair_sphere()
    A = torch.tensor(s.A, device="cuda")
    B = torch.tensor(s.B, device="cuda")
    rng = np.random.default_rng(8)
    rots = np.concatenate([np.eye(3)[None], synth.random_rotations(rng, 3)])
    k = len(rots)
    R0 = np.repeat(s.R0, k, axis=0)
    E, G, st = ctx.tcm_gradients_batch([(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int),
                                       np.full(k, s.L), R0, rotB=rots, precision=tcm.TCM_FP64)
    E2, _ = ctx.tcm_energy_batch([(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int),
                                 np.full(k, s.L), R0, rotB=rots, precision=tcm.TCM_FP64)
    torch.cuda.synchronize()
    assert bool(torch.all(st == 0)) and torch.equal(E, E2)
    G = G.cpu().numpy()
    cA, _ = oracle.center_radius(s.A)
    cB, _ = oracle.center_radius(s.B)
    for i in range(k):
        Eo, F, tA, tB, SF = oracle_grads(s.A, cA, s.B, cB, s.L, R0[i], rots[i])
        e = errors(G[i], F, tA, tB, SF, R0[i], mixed=False)
        print(f"orientation {i}: force {e[0]:.2e}, torque A {e[1]:.2e}, torque B {e[2]:.2e}")
        assert max(e) < TOL_FP64, e
        bal = G[i, 3:6] + G[i, 6:] + np.cross(R0[i], G[i, :3])
        assert np.linalg.norm(bal) < 1e-12 * np.linalg.norm(R0[i]) * SF


@pytest.mark.parametrize("L", [0, 1, 2, 9, 24])
def test_degrees_and_directions_fp64(ctx, tcm, L):
    rng = np.random.default_rng(40 + L)
    A = synth.pack(synth.uniform_ball(rng, 300, 5.0), synth.charges_uniform_net_zero(rng, 300))
    B = synth.pack(synth.uniform_ball(rng, 250, 4.0), synth.charges_uniform_net_zero(rng, 250))
    A[:, 3] += 0.05  # nonzero monopoles too (the L = 0 force is their product)
    B[:, 3] -= 0.04
    dirs = np.array([[0, 0, 1.0], [0, 0, -1.0], [1e-9, 0, 1.0], [0.3, -0.4, 0.5], [-1.0, 0.0, 0.0]])
    R0 = dirs / np.linalg.norm(dirs, axis=1)[:, None] * 25.0
    k = len(R0)
    rot = synth.random_rotations(rng, k)
    E, G, st = ctx.tcm_gradients_batch([(torch.tensor(A, device="cuda"), None, None),
                                        (torch.tensor(B, device="cuda"), None, None)],
                                       np.zeros(k, int), np.ones(k, int), np.full(k, L), R0, rotB=rot,
                                       precision=tcm.TCM_FP64)
    torch.cuda.synchronize()
    G = G.cpu().numpy()
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    for i in range(k):
        Eo, F, tA, tB, SF = oracle_grads(A, cA, B, cB, L, R0[i], rot[i])
        e = errors(G[i], F, tA, tB, SF, R0[i], mixed=False)
        assert max(e) < TOL_FP64, (i, e)


@pytest.mark.parametrize("rotate_cached", [False, True])
def test_mixed_batch_forces_and_torques(tcm, rotate_cached):
    s = synth.protein_pes_scan(n=8000, n_orient=32, radius=22.0, r_lo=55.0, r_hi=110.0, L=20)
    A = torch.tensor(s.A, dtype=torch.float32, device="cuda")
    B = torch.tensor(s.B, dtype=torch.float32, device="cuda")
    ctx = tcm.Context(lmax_cap=24)
    try:
        systems = [(A, None, None), (B, None, None)]
        if rotate_cached:
            mA = ctx.tcm_moments(A, 20, precision=tcm.TCM_MIXED)
            mB = ctx.tcm_moments(B, 20, precision=tcm.TCM_MIXED)
            systems = [tcm.make_system(A, mA.center, mA.radius, moments=mA),
                       tcm.make_system(B, mB.center, mB.radius, moments=mB)]
            ctx.tcm_ctx_set_rotate_cached(True)
        k = len(s.R0)
        E, G, st = ctx.tcm_gradients_batch(systems, np.zeros(k, int), np.ones(k, int), np.full(k, s.L), s.R0,
                                           rotB=s.rotB, precision=tcm.TCM_MIXED)
        torch.cuda.synchronize()
        assert bool(torch.all(st == 0))
        G = G.cpu().numpy()
        Af = s.A.astype(np.float32).astype(np.float64)
        Bf = s.B.astype(np.float32).astype(np.float64)
        cA, _ = oracle.center_radius(Af)
        cB, _ = oracle.center_radius(Bf)
        rep = MixedEnergyReport("mixed forces and torques")
        for i in (0, 13, 31):
            Eo, F, tA, tB, SF = oracle_grads(Af, cA, Bf, cB, s.L, s.R0[i], s.rotB[i])
            R = np.linalg.norm(s.R0[i])
            rep.add_vec(G[i][:3], F, SF, f"orientation {i}, force on B")
            rep.add_vec(G[i][3:6], tA, R * SF, f"orientation {i}, torque on A")
            rep.add_vec(G[i][6:], tB, R * SF, f"orientation {i}, torque on B")
        rep.check()
    finally:
        ctx.close()


def test_not_converged_item_gives_nan_gradients(ctx, tcm):
    rng = np.random.default_rng(3)
    A = torch.tensor(synth.pack(synth.uniform_ball(rng, 100, 5.0), synth.charges_uniform_net_zero(rng, 100)),
                     device="cuda")
    R0 = np.array([[0.0, 0.0, 30.0], [0.0, 0.0, 2.0]])  # the second violates Eq. (mainCond)
    E, G, st = ctx.tcm_gradients_batch([(A, None, None)], [0, 0], [0, 0], [6, 6], R0, precision=tcm.TCM_FP64,
                                       rotB=np.stack([np.eye(3)] * 2))
    # host-known radius? not here (computed on the device), so the item comes back flagged
    torch.cuda.synchronize()
    assert st.tolist() == [0, tcm.TCM_ENOTCONV]
    assert bool(torch.all(torch.isfinite(G[0]))) and bool(torch.all(torch.isnan(G[1])))
