"""Eq. (Formula) through the three ways the contraction kernel receives B's moments: in the lab
frame (rotated into the frame of R0 inside the kernel, like A's), already in that frame (the frame
rotation folded into B's atom transform), and rotated from B's moment cache.  Degrees 0 to 24 and
separations along +z, -z, 1e-9 rad off +z, a generic direction and -x put the frame's angles at
their edges (beta = 0 and pi, an azimuth that is undefined on the axis); the identity and random
rotations of B; double precision against the oracle at the 1e-12 bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import TOL_FP64, energy_error

pytestmark = pytest.mark.gpu

DIRS = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [1e-9, 0.0, 1.0], [0.3, -0.4, 0.5], [-1.0, 0.0, 0.0]])


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
def systems():
    rng = np.random.default_rng(77)
    A = synth.pack(synth.uniform_ball(rng, 150, 4.0), synth.charges_uniform_net_zero(rng, 150))
    B = synth.pack(synth.uniform_ball(rng, 120, 3.5), synth.charges_uniform_net_zero(rng, 120))
    A[:, 3] += 0.03  # charged systems: the monopole terms take part as well
    B[:, 3] -= 0.02
    return A, B


@pytest.mark.parametrize("L", [0, 1, 2, 3, 7, 12, 24])
def test_contraction_modes_fp64(tcm, systems, L):
    A, B = systems
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    R0 = DIRS / np.linalg.norm(DIRS, axis=1)[:, None] * 20.0
    k = len(R0)
    rots = synth.random_rotations(np.random.default_rng(100 + L), k)
    rots[0] = np.eye(3)
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    ctx = tcm.Context(lmax_cap=24)
    try:
        mA = ctx.tcm_moments(Ad, 24, precision=tcm.TCM_FP64)
        mB = ctx.tcm_moments(Bd, 24, precision=tcm.TCM_FP64)
        cached = [tcm.make_system(Ad, mA.center, mA.radius, moments=mA),
                  tcm.make_system(Bd, mB.center, mB.radius, moments=mB)]
        plain = [(Ad, None, None), (Bd, None, None)]
        a, b, Ls = np.zeros(k, int), np.ones(k, int), np.full(k, L)
        E_lab, s1 = ctx.tcm_energy_batch(plain, a, b, Ls, R0, precision=tcm.TCM_FP64)
        E_frame, s2 = ctx.tcm_energy_batch(plain, a, b, Ls, R0, rotB=rots, precision=tcm.TCM_FP64)
        ctx.tcm_ctx_set_rotate_cached(True)
        E_rot, s3 = ctx.tcm_energy_batch(cached, a, b, Ls, R0, rotB=rots, precision=tcm.TCM_FP64)
        torch.cuda.synchronize()
        for st in (s1, s2, s3):
            assert bool(torch.all(st == 0))
        QA = oracle.moments(A, cA, L)
        QB = oracle.moments(B, cB, L)
        worst = 0.0
        for i in range(k):
            Eo = oracle.tcm_energy(L, QA, QB, R0[i])
            e1 = energy_error(float(E_lab[i]), Eo, oracle.tcm_blocks(L, QA, QB, R0[i]))
            QBr = oracle.moments(B, cB, L, rot=rots[i])
            Eo = oracle.tcm_energy(L, QA, QBr, R0[i])
            blocks = oracle.tcm_blocks(L, QA, QBr, R0[i])
            e2 = energy_error(float(E_frame[i]), Eo, blocks)
            e3 = energy_error(float(E_rot[i]), Eo, blocks)
            worst = max(worst, e1, e2, e3)
            assert max(e1, e2, e3) < TOL_FP64, (L, i, e1, e2, e3)
        print(f"L={L}: worst error over the three modes {worst:.2e}")
    finally:
        ctx.close()


@pytest.mark.parametrize("L", [1, 7, 24])
def test_gradient_modes_agree_fp64(tcm, systems, L):
    """Forces and torques of the same placements through the three modes (the in-frame mode is
    checked against the oracle's derivatives in test_gpu_gradients.py): the rotate-from-cache
    mode must give the in-frame values, and the lab mode those of the identity rotation."""
    A, B = systems
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    R0 = DIRS / np.linalg.norm(DIRS, axis=1)[:, None] * 20.0
    k = len(R0)
    rots = synth.random_rotations(np.random.default_rng(200 + L), k)
    eye = np.stack([np.eye(3)] * k)
    ctx = tcm.Context(lmax_cap=24)
    try:
        mA = ctx.tcm_moments(Ad, 24, precision=tcm.TCM_FP64)
        mB = ctx.tcm_moments(Bd, 24, precision=tcm.TCM_FP64)
        cached = [tcm.make_system(Ad, mA.center, mA.radius, moments=mA),
                  tcm.make_system(Bd, mB.center, mB.radius, moments=mB)]
        plain = [(Ad, None, None), (Bd, None, None)]
        a, b, Ls = np.zeros(k, int), np.ones(k, int), np.full(k, L)
        _, G_lab, s1 = ctx.tcm_gradients_batch(plain, a, b, Ls, R0, precision=tcm.TCM_FP64)
        _, G_id, s2 = ctx.tcm_gradients_batch(plain, a, b, Ls, R0, rotB=eye, precision=tcm.TCM_FP64)
        _, G_frame, s3 = ctx.tcm_gradients_batch(plain, a, b, Ls, R0, rotB=rots, precision=tcm.TCM_FP64)
        ctx.tcm_ctx_set_rotate_cached(True)
        _, G_rot, s4 = ctx.tcm_gradients_batch(cached, a, b, Ls, R0, rotB=rots, precision=tcm.TCM_FP64)
        torch.cuda.synchronize()
        for st in (s1, s2, s3, s4):
            assert bool(torch.all(st == 0))
        G_lab, G_id, G_frame, G_rot = (g.cpu().numpy() for g in (G_lab, G_id, G_frame, G_rot))
        for i in range(k):
            for part in (slice(0, 3), slice(3, 6), slice(6, 9)):
                for x, ref in ((G_lab[i, part], G_id[i, part]), (G_rot[i, part], G_frame[i, part])):
                    scale = max(np.linalg.norm(ref), 1e-3 * np.abs(G_frame[i]).max(), 1e-300)
                    assert np.linalg.norm(x - ref) / scale < TOL_FP64 * 10, (L, i, part, x, ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_does_not_depend_on_the_batch(tcm, systems, precision):
    """The contraction kernel's CTA size follows the batch (its largest degree and its item count),
    so the same item must give the same bits alone, beside a degree-24 item, and in a batch of
    more than a thousand items; energies and gradients alike."""
    A, B = systems
    prec = tcm.TCM_FP64 if precision == "fp64" else tcm.TCM_MIXED
    dt = torch.float64 if precision == "fp64" else torch.float32
    T = [(torch.tensor(A, dtype=dt, device="cuda"), None, None), (torch.tensor(B, dtype=dt, device="cuda"), None, None)]
    rng = np.random.default_rng(5)
    n = 1100
    R0 = synth.unit_vectors(rng, n) * rng.uniform(12.0, 20.0, n)[:, None]
    rot = synth.random_rotations(rng, n)
    L = np.where(np.arange(n) % 2 == 0, 20, 8)
    L[1] = 24
    ia, ib = np.zeros(n, int), np.ones(n, int)
    with tcm.Context(lmax_cap=24) as ctx:
        E_all, _ = ctx.tcm_energy_batch(T, ia, ib, L, R0, rotB=rot, precision=prec)
        Eg_all, G_all, _ = ctx.tcm_gradients_batch(T, ia, ib, L, R0, rotB=rot, precision=prec)
        for k in (0, 2, 3):  # L = 20, 20, 8
            for sel in ([k], [k, 1]):  # alone; beside the degree-24 item
                E1, _ = ctx.tcm_energy_batch(T, ia[sel], ib[sel], L[sel], R0[sel], rotB=rot[sel], precision=prec)
                Eg1, G1, _ = ctx.tcm_gradients_batch(T, ia[sel], ib[sel], L[sel], R0[sel], rotB=rot[sel],
                                                     precision=prec)
                torch.cuda.synchronize()
                assert float(E1[0]) == float(E_all[k]), (k, sel, float(E1[0]) - float(E_all[k]))
                assert float(Eg1[0]) == float(E_all[k]) == float(Eg_all[k])
                assert torch.equal(G1[0], G_all[k]), (k, sel)
