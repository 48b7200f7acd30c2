"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element
on the same seeded inputs (tolerances in tcm_testlib)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import (TOL_FP64, TOL_MIX_E, TOL_MIX_MOM, MixedEnergyReport, degree_scales, energy_error,
                         moment_error, oracle_moments_threaded)

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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def sphere_system(seed, n, radius=5.0, shift=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    S = synth.pack(synth.uniform_ball(rng, n, radius), synth.charges_uniform_net_zero(rng, n) if n > 1 else np.ones(n))
    S[:, :3] += shift
    return S


# ----------------------------------------------------------------------------- moments

@pytest.mark.parametrize("n", [1, 31, 33, 1025, 4100, 9000])
@pytest.mark.parametrize("L", [0, 1, 2, 7, 10, 13, 20, 24])
def test_moments_fp64_vs_oracle(ctx, tcm, n, L):
    S = sphere_system(100 + n, n, shift=(3.0, -1.0, 2.0))
    c, a = oracle.center_radius(S)
    m = ctx.tcm_moments(dev(S), L, precision=tcm.TCM_FP64)
    assert np.allclose(m.center, c, rtol=0, atol=1e-12) and abs(m.radius - a) < 1e-12
    ref = oracle_moments_threaded(S, c, L)
    err = moment_error(tcm.unpack(m.q), ref, degree_scales(S, c, L))
    assert err < TOL_FP64, err


@pytest.mark.parametrize("n", [1, 31, 33, 1025, 4100, 9000])
@pytest.mark.parametrize("L", [0, 1, 2, 7, 10, 13, 20, 24])
def test_moments_mixed_vs_oracle(ctx, tcm, n, L):
    S = sphere_system(200 + n, n, shift=(-2.0, 0.5, 7.0))
    c, a = oracle.center_radius(S)
    m = ctx.tcm_moments(dev(S), L, precision=tcm.TCM_MIXED)
    ref = oracle_moments_threaded(S, c, L)
    err = moment_error(tcm.unpack(m.q), ref, degree_scales(S, c, L))
    assert err < TOL_MIX_MOM, err


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_mixed_low_degrees_to_double_accuracy(ctx, tcm, dtype):
    """Degrees l <= 2 of the mixed path come from float-float Cartesian sums about the centre,
    rotated in double: they match the oracle to double accuracy, not to the float recurrence's."""
    S = sphere_system(77, 40000, radius=20.0, shift=(50.0, -20.0, 10.0))
    Sx = S.astype(np.float32).astype(np.float64) if dtype == "float32" else S
    rot = synth.random_rotations(np.random.default_rng(3), 1)[0]
    m = ctx.tcm_moments(dev(Sx, getattr(torch, dtype)), 6, precision=tcm.TCM_MIXED, rot=rot)
    ref = oracle_moments_threaded(Sx, m.center, 6, rot=rot)
    q = tcm.unpack(m.q)
    sc = degree_scales(Sx, m.center, 6, rot=rot)
    for l in range(3):
        sl = slice(l * l, (l + 1) * (l + 1))
        err = np.max(np.abs(q[sl] - ref[sl])) / max(np.linalg.norm(ref[sl]), 1e-3 * sc[l])
        assert err < 1e-11, (l, err)
    assert moment_error(q, ref, sc) < TOL_MIX_MOM


@pytest.mark.parametrize("precision", [0, 1])
def test_moments_float32_coordinates_rotation_given_centre(ctx, tcm, precision):
    rng = np.random.default_rng(5)
    S = sphere_system(7, 3000, radius=20.0, shift=(100.0, -50.0, 25.0))
    S32 = S.astype(np.float32).astype(np.float64)  # what the float32 input holds
    rot = synth.random_rotations(rng, 1)[0]
    cgiv = np.array([99.5, -50.25, 24.75])
    L = 16
    m = ctx.tcm_moments(dev(S32, torch.float32), L, precision=precision, rot=rot, center=cgiv, radius=25.0)
    assert np.allclose(m.center, cgiv) and m.radius == 25.0
    ref = oracle_moments_threaded(S32, cgiv, L, rot=rot)
    err = moment_error(tcm.unpack(m.q), ref, degree_scales(S32, cgiv, L, rot=rot))
    assert err < (TOL_FP64 if precision == 0 else TOL_MIX_MOM), err


def test_moments_empty_and_single_charge_at_centre(ctx, tcm):
    empty = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    m = ctx.tcm_moments(empty, 6, precision=tcm.TCM_MIXED, center=(0, 0, 0), radius=1.0)
    assert torch.all(m.q == 0)
    one = dev(np.array([[1.0, 2.0, 3.0, 0.75]]))
    for prec in (0, 1):
        m = ctx.tcm_moments(one, 8, precision=prec)  # centroid = the charge itself, radius 0
        q = m.q.cpu().numpy()
        assert q[0] == 0.75 and np.all(q[1:] == 0.0)


# ----------------------------------------------------------------------------- energies

def test_single_pair_fp64_energy_and_direct(ctx, tcm):
    """Single-pair workload: 2 x 200 charges in r = 10 A spheres, R0 = 40 A, Lmax = 10, FP64."""
    s = synth.single_pair_sphere()
    A, B = dev(s.A), dev(s.B)
    ma = ctx.tcm_moments(A, s.L, precision=tcm.TCM_FP64)
    mb = ctx.tcm_moments(B, s.L, precision=tcm.TCM_FP64)
    R0 = s.R0[0]
    E = ctx.tcm_energy(ma, mb, R0, s.L)
    cA, _ = oracle.center_radius(s.A)
    cB, _ = oracle.center_radius(s.B)
    QA, QB = oracle.moments(s.A, cA, s.L), oracle.moments(s.B, cB, s.L)
    Eo = oracle.tcm_energy(s.L, QA, QB, R0)
    blocks = oracle.tcm_blocks(s.L, QA, QB, R0)
    assert energy_error(E, Eo, blocks) < TOL_FP64
    Ed = ctx.tcm_direct(A, B, R0)
    Edo, scale = oracle.direct(s.A, cA, s.B, cB, R0, return_abs=True)
    assert abs(Ed - Edo) / scale < TOL_FP64
    # the batched path at FP64 gives the same energy
    Eb, st = ctx.tcm_energy_batch([(A, None, None), (B, None, None)], [0], [1], [s.L], R0[None], precision=tcm.TCM_FP64)
    torch.cuda.synchronize()
    assert int(st[0]) == 0 and energy_error(float(Eb[0]), Eo, blocks) < TOL_FP64


def test_protein_pes_scan_full_size_every_orientation(ctx, tcm):
    """Protein-like PES scan at full size (2 x 20,000 atoms, 256 orientations, L = 20), mixed
    precision, the launch the benchmark times; the oracle on every orientation."""
    s = synth.protein_pes_scan()
    A, B = dev(s.A, torch.float32), dev(s.B, torch.float32)
    k = len(s.R0)
    E, st = ctx.tcm_energy_batch([(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int),
                                 np.full(k, s.L), s.R0, rotB=s.rotB, precision=tcm.TCM_MIXED)
    torch.cuda.synchronize()
    assert torch.all(st == 0)
    E = E.cpu().numpy()
    Af, Bf = s.A.astype(np.float32).astype(np.float64), s.B.astype(np.float32).astype(np.float64)
    cA, _ = oracle.center_radius(Af)
    cB, _ = oracle.center_radius(Bf)
    QA = oracle_moments_threaded(Af, cA, s.L)
    rep = MixedEnergyReport("protein-like scan, 256 orientations")
    for kk in range(k):
        QB = oracle_moments_threaded(Bf, cB, s.L, rot=s.rotB[kk])
        rep.add(float(E[kk]), oracle.tcm_energy(s.L, QA, QB, s.R0[kk]), oracle.tcm_blocks(s.L, QA, QB, s.R0[kk]),
                f"orientation {kk}")
    rep.check()


def test_batch_alone_vs_in_mix_and_repeatability(ctx, tcm):
    """Each item's result is independent of the rest of the batch, and runs repeat bitwise."""
    rng = np.random.default_rng(17)
    systems = [sphere_system(300 + i, int(n), radius=float(r)) for i, (n, r) in
               enumerate([(500, 6.0), (3000, 9.0), (12000, 15.0), (80, 3.0), (7000, 12.0)])]
    T = [(dev(S, torch.float32), None, None) for S in systems]
    rad = [oracle.center_radius(S)[1] for S in systems]
    items = [(0, 1, 12), (2, 3, 24), (1, 4, 8), (4, 2, 16), (3, 0, 10)]
    a = [i[0] for i in items]
    b = [i[1] for i in items]
    L = [i[2] for i in items]
    R0 = np.array([synth.unit_vectors(rng, 1)[0] * 1.7 * (rad[i] + rad[j]) for i, j, _ in items])
    rot = synth.random_rotations(rng, len(items))
    E_mix, _ = ctx.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=tcm.TCM_MIXED)
    E_mix2, _ = ctx.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=tcm.TCM_MIXED)
    torch.cuda.synchronize()
    assert torch.equal(E_mix, E_mix2)
    for k in range(len(items)):
        E1, _ = ctx.tcm_energy_batch(T, [a[k]], [b[k]], [L[k]], R0[k:k + 1], rotB=rot[k:k + 1], precision=tcm.TCM_MIXED)
        torch.cuda.synchronize()
        assert float(E1[0]) == float(E_mix[k])
    # and each is right
    rep = MixedEnergyReport("alone-vs-mix batch")
    for k in range(len(items)):
        Sa, Sb = systems[a[k]].astype(np.float32).astype(np.float64), systems[b[k]].astype(np.float32).astype(np.float64)
        ca, cb = oracle.center_radius(Sa)[0], oracle.center_radius(Sb)[0]
        QA = oracle_moments_threaded(Sa, ca, L[k])
        QB = oracle_moments_threaded(Sb, cb, L[k], rot=rot[k])
        rep.add(float(E_mix[k]), oracle.tcm_energy(L[k], QA, QB, R0[k]), oracle.tcm_blocks(L[k], QA, QB, R0[k]),
                f"item {k}")
    rep.check()


# ----------------------------------------------------------------------------- error paths

def test_not_converged_paths(ctx, tcm):
    S = sphere_system(11, 100, radius=5.0)
    A = dev(S)
    m = ctx.tcm_moments(A, 4, precision=tcm.TCM_FP64)
    with pytest.raises(tcm.TcmError) as e:
        ctx.tcm_energy(m, m, [0.0, 0.0, 1.5 * m.radius], 4)
    assert e.value.code == tcm.TCM_ENOTCONV
    # host-known radii: rejected before any work
    with pytest.raises(tcm.TcmError) as e:
        ctx.tcm_energy_batch([(A, m.center, m.radius)], [0], [0], [4], [[0.0, 0.0, 1.0]])
    assert e.value.code == tcm.TCM_ENOTCONV
    # radii computed on the device: NaN and a per-item status
    E, st = ctx.tcm_energy_batch([(A, None, None)], [0, 0], [0, 0], [4, 4],
                                 [[0.0, 0.0, 1.0], [0.0, 0.0, 3.0 * m.radius]])
    torch.cuda.synchronize()
    assert int(st[0]) == tcm.TCM_ENOTCONV and np.isnan(float(E[0]))
    assert int(st[1]) == tcm.TCM_OK and np.isfinite(float(E[1]))


def test_invalid_arguments(ctx, tcm):
    S = dev(sphere_system(12, 64))
    with pytest.raises(tcm.TcmError) as e:
        ctx.tcm_moments(S, 25)
    assert e.value.code == tcm.TCM_EINVAL
    raw = torch.zeros(4 * 64 + 1, dtype=torch.float32, device="cuda")
    mis = raw[1:].view(64, 4)  # 4-byte offset: not 16-byte aligned
    with pytest.raises(tcm.TcmError) as e:
        ctx.tcm_moments(mis, 4)
    assert e.value.code == tcm.TCM_EINVAL
    with pytest.raises(tcm.TcmError) as e:
        ctx.tcm_energy_batch([(S, None, None)], [0], [3], [4], [[0.0, 0.0, 100.0]])
    assert e.value.code == tcm.TCM_EINVAL


@pytest.mark.parametrize("precision_name", ["TCM_FP64", "TCM_MIXED"])
def test_degenerate_batch(ctx, tcm, precision_name):
    """Empty systems, single charges at the centre, all-zero charges, Lmax = 0 and Lmax = 24
    items side by side in one batch: each against the oracle (or its closed form)."""
    precision = getattr(tcm, precision_name)
    rng = np.random.default_rng(21)
    empty = np.zeros((0, 4))
    one = np.array([[1.0, -2.0, 0.5, 0.8]])
    zeros = synth.pack(synth.uniform_ball(rng, 500, 4.0), np.zeros(500))
    gen = sphere_system(22, 700, radius=5.0)
    gen[:, 3] += 0.01
    systems = [empty, one, zeros, gen]
    dt = torch.float64 if precision == tcm.TCM_FP64 else torch.float32
    T = [(dev(S, dt) if len(S) else torch.zeros((0, 4), dtype=dt, device="cuda"),
          np.zeros(3) if len(S) == 0 else None, None) for S in systems]
    items = [(0, 3, 6), (1, 3, 0), (1, 3, 24), (2, 3, 10), (3, 1, 12), (1, 1, 4), (3, 3, 24)]
    a, b, L = zip(*items)
    R0 = np.array([[0.0, 0.0, 40.0], [30.0, 1.0, -2.0], [0.0, 35.0, 0.0], [25.0, 25.0, 25.0],
                   [-20.0, 10.0, 30.0], [5.0, 0.0, 0.0], [1e-9, 0.0, -30.0]])
    E, st = ctx.tcm_energy_batch(T, a, b, L, R0, precision=precision)
    torch.cuda.synchronize()
    assert st.tolist() == [0] * len(items)
    E = E.cpu().numpy()
    mixed = precision == tcm.TCM_MIXED
    rep = MixedEnergyReport("degenerate batch")
    for k, (ia, ib, Lk) in enumerate(items):
        Sa = systems[ia].astype(np.float32).astype(np.float64) if mixed else systems[ia]
        Sb = systems[ib].astype(np.float32).astype(np.float64) if mixed else systems[ib]
        ca = np.zeros(3) if len(Sa) == 0 else oracle.center_radius(Sa)[0]
        cb = np.zeros(3) if len(Sb) == 0 else oracle.center_radius(Sb)[0]
        QA = oracle.moments(Sa, ca, Lk) if len(Sa) else np.zeros((Lk + 1) ** 2, dtype=complex)
        QB = oracle.moments(Sb, cb, Lk) if len(Sb) else np.zeros((Lk + 1) ** 2, dtype=complex)
        Eo = oracle.tcm_energy(Lk, QA, QB, R0[k])
        blocks = oracle.tcm_blocks(Lk, QA, QB, R0[k])
        if not np.any(blocks):
            assert E[k] == 0.0, (k, E[k])
        elif mixed:
            rep.add(E[k], Eo, blocks, f"item {k}")
        else:
            assert energy_error(E[k], Eo, blocks) < TOL_FP64, (k, E[k], Eo)
    if mixed:
        rep.check()
    # a single charge at its own centroid against itself: q^2 / R exactly at every Lmax
    assert abs(E[5] - 0.8 * 0.8 / 5.0) <= 1e-15 * 0.128 * (1 if not mixed else 1e8)


@pytest.mark.parametrize("n", [0, 1, 100, 5000, 32768, 32769, 70000])
def test_prepare_float32_centre_and_radius(ctx, tcm, n):
    """Step a1 for float32 systems: one cluster per system up to 32,768 atoms (float arithmetic
    with an error-free centroid sum and an exact double radius over the float-filtered
    candidates), the tiled kernels above: both against the oracle on the same float values."""
    rng = np.random.default_rng(300 + n)
    S = synth.pack(synth.uniform_ball(rng, n, 25.0) + [1000.0, -500.0, 250.0], rng.normal(size=n))
    S32 = S.astype(np.float32).astype(np.float64)
    t = torch.tensor(S32, dtype=torch.float32, device="cuda") if n else torch.zeros((0, 4), device="cuda")
    c, a = ctx.tcm_prepare(t)
    if n == 0:
        assert a == 0.0
        return
    c_ref, a_ref = oracle.center_radius(S32)
    assert np.allclose(c, c_ref, rtol=0, atol=1e-12 * 1000.0), (c, c_ref)
    assert abs(a - a_ref) <= 1e-12 * a_ref, (a, a_ref)
