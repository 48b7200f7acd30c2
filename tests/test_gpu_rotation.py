"""Wigner rotation of cached moments (tcm_rotate_moments and the batched rotate-from-cache mode)
against the oracle's moments of the rotated atoms, Eq. (multipole) evaluated on R x: the rotation
of the moments is checked against the definition, not against another rotation routine."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import (TOL_FP64, TOL_MIX_MOM, MixedEnergyReport, degree_scales, energy_error, moment_error,
                         oracle_moments_threaded)

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


def rot_axis(axis, ang):
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def special_rotations():
    rng = np.random.default_rng(77)
    out = {"identity": np.eye(3), "z_only": rot_axis([0, 0, 1], 0.7), "pi_about_x": rot_axis([1, 0, 0], np.pi),
           "pi_about_xy": rot_axis([1, 1, 0], np.pi), "tiny_beta": rot_axis([1, 2, 0.3], 1e-9),
           "near_pi_beta": rot_axis([0.3, 1, 0], np.pi - 1e-9), "half_pi_y": rot_axis([0, 1, 0], np.pi / 2)}
    for i, R in enumerate(synth.random_rotations(rng, 4)):
        out[f"random{i}"] = R
    return out


def system(seed, n, radius):
    rng = np.random.default_rng(seed)
    return synth.pack(synth.random_walk(rng, n, radius) + [4.0, -3.0, 1.0], synth.charges_normal_net_zero(rng, n))


@pytest.mark.parametrize("L", [0, 1, 5, 16, 24])
def test_rotate_fp64_moments_vs_oracle_rotated_atoms(ctx, tcm, L):
    S = system(3 + L, 3000, 18.0)
    c, _ = oracle.center_radius(S)
    m = ctx.tcm_moments(torch.tensor(S, device="cuda"), L, precision=tcm.TCM_FP64)
    rots = special_rotations()
    names = list(rots)
    outs = ctx.tcm_rotate_moments([m] * len(names), np.stack([rots[k] for k in names]))
    torch.cuda.synchronize()
    for name, o in zip(names, outs):
        ref = oracle_moments_threaded(S, c, L, rot=rots[name])
        err = moment_error(tcm.unpack(o.q), ref, degree_scales(S, c, L, rot=rots[name]))
        assert err < TOL_FP64, (name, err)
        assert np.allclose(o.center, m.center) and o.radius == m.radius


def test_rotate_lower_degree_and_in_place(ctx, tcm):
    S = system(11, 5000, 20.0)
    c, _ = oracle.center_radius(S)
    m = ctx.tcm_moments(torch.tensor(S, device="cuda"), 20, precision=tcm.TCM_FP64)
    R = synth.random_rotations(np.random.default_rng(5), 2)
    low = ctx.tcm_rotate_moments(m, R[0], lmax=9)
    assert low.lmax == 9 and low.q.numel() == 100
    ref = oracle_moments_threaded(S, c, 9, rot=R[0])
    assert moment_error(tcm.unpack(low.q), ref, degree_scales(S, c, 9, rot=R[0])) < TOL_FP64
    # composition in place: R1 after R0 equals the single rotation R1 R0
    q0 = m.q.clone()
    ctx.tcm_rotate_moments(m, R[0], out=m)
    ctx.tcm_rotate_moments(m, R[1], out=m)
    torch.cuda.synchronize()
    ref = oracle_moments_threaded(S, c, 20, rot=R[1] @ R[0])
    assert moment_error(tcm.unpack(m.q), ref, degree_scales(S, c, 20, rot=R[1] @ R[0])) < TOL_FP64
    assert not torch.equal(q0, m.q)


def test_rotate_mixed_moments(ctx, tcm):
    S = system(12, 20000, 30.0)
    c, _ = oracle.center_radius(S.astype(np.float32).astype(np.float64))
    m = ctx.tcm_moments(torch.tensor(S, dtype=torch.float32, device="cuda"), 20, precision=tcm.TCM_MIXED)
    S32 = S.astype(np.float32).astype(np.float64)
    for name, R in special_rotations().items():
        o = ctx.tcm_rotate_moments(m, R)
        ref = oracle_moments_threaded(S32, m.center, 20, rot=R)
        err = moment_error(tcm.unpack(o.q), ref, degree_scales(S32, m.center, 20, rot=R))
        assert err < TOL_MIX_MOM, (name, err)


def test_rotate_invalid_arguments(ctx, tcm):
    S = system(13, 100, 6.0)
    m = ctx.tcm_moments(torch.tensor(S, device="cuda"), 6, precision=tcm.TCM_FP64)
    with pytest.raises(tcm.TcmError):
        ctx.tcm_rotate_moments(m, np.eye(3), lmax=7)  # above the input's lmax
    with pytest.raises(tcm.TcmError):
        ctx.tcm_rotate_moments(m, np.full((3, 3), np.nan))
    with pytest.raises(tcm.TcmError):
        ctx.tcm_rotate_moments([m, m], np.eye(3))  # one rotation for two sets


@pytest.mark.parametrize("precision_name", ["TCM_FP64", "TCM_MIXED"])
def test_batch_rotated_sides_from_cache(tcm, precision_name):
    """PES-scan shaped batch (B rotated per orientation) with B's moments rotated from its cache,
    against the oracle on the rotated atoms and against the recomputed path."""
    precision = getattr(tcm, precision_name)
    s = synth.protein_pes_scan(n=6000, n_orient=48, radius=20.0, r_lo=50.0, r_hi=100.0, L=20)
    dt = torch.float64 if precision == tcm.TCM_FP64 else torch.float32
    A = torch.tensor(s.A, dtype=dt, device="cuda")
    B = torch.tensor(s.B, dtype=dt, device="cuda")
    ctx = tcm.Context(lmax_cap=24)
    try:
        mA = ctx.tcm_moments(A, s.L, precision=precision)
        mB = ctx.tcm_moments(B, s.L, precision=precision)
        sysA = tcm.make_system(A, mA.center, mA.radius, moments=mA)
        sysB = tcm.make_system(B, mB.center, mB.radius, moments=mB)
        k = len(s.R0)
        a, b, L = np.zeros(k, int), np.ones(k, int), np.full(k, s.L)
        E_re, _ = ctx.tcm_energy_batch([sysA, sysB], a, b, L, s.R0, rotB=s.rotB, precision=precision)
        ctx.tcm_ctx_set_rotate_cached(True)
        E_ro, st = ctx.tcm_energy_batch([sysA, sysB], a, b, L, s.R0, rotB=s.rotB, precision=precision)
        torch.cuda.synchronize()
        assert bool(torch.all(st == 0))
        Af = s.A.astype(np.float32).astype(np.float64) if precision == tcm.TCM_MIXED else s.A
        Bf = s.B.astype(np.float32).astype(np.float64) if precision == tcm.TCM_MIXED else s.B
        QA = oracle_moments_threaded(Af, mA.center, s.L)
        worst = 0.0
        mixed = precision == tcm.TCM_MIXED
        rep = MixedEnergyReport("rotated from the cache and recomputed")
        for i in (0, 17, 47):
            QB = oracle_moments_threaded(Bf, mB.center, s.L, rot=s.rotB[i])
            Eo = oracle.tcm_energy(s.L, QA, QB, s.R0[i])
            blocks = oracle.tcm_blocks(s.L, QA, QB, s.R0[i])
            if mixed:
                rep.add(float(E_ro[i]), Eo, blocks, f"orientation {i}, rotated from the cache")
                rep.add(float(E_re[i]), Eo, blocks, f"orientation {i}, recomputed")
            else:
                worst = max(worst, energy_error(float(E_ro[i]), Eo, blocks))
                assert energy_error(float(E_re[i]), Eo, blocks) < TOL_FP64
        if mixed:
            rep.check()
        else:
            print(f"rotate-from-cache energy error {worst:.3e}")
            assert worst < TOL_FP64
    finally:
        ctx.close()
