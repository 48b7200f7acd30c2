"""GPU parity at the full sizes of the larger workloads, through the batched C ABI call, with
the oracle on sampled items (tolerances in tcm_testlib)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import TOL_FP64, MixedEnergyReport, energy_error, oracle_moments_threaded

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


def f32(a):
    return a.astype(np.float32).astype(np.float64)


def check_items(name, sysA, sysB, rot, R0, L, E, sample):
    rep = MixedEnergyReport(name)
    for k in sample:
        A, B = f32(sysA(k)), f32(sysB(k))
        cA, _ = oracle.center_radius(A)
        cB, _ = oracle.center_radius(B)
        QA = oracle_moments_threaded(A, cA, L[k])
        QB = oracle_moments_threaded(B, cB, L[k], rot=rot[k])
        rep.add(float(E[k]), oracle.tcm_energy(L[k], QA, QB, R0[k]), oracle.tcm_blocks(L[k], QA, QB, R0[k]),
                f"item {k} (L={L[k]}, N=({len(A)},{len(B)}))")
    rep.check()


def uneven_sample(b, per_cell=2):
    """Items of every degree in every decile of the pair size (N_A + N_B): per_cell each."""
    n = np.array([len(s) for s in b.systems])
    sizes = n[b.pair_a] + n[b.pair_b]
    edges = np.quantile(sizes, np.linspace(0, 1, 11))
    sample = []
    for L in sorted(set(int(x) for x in b.L)):
        for d in range(10):
            idx = np.where((b.L == L) & (sizes >= edges[d]) & (sizes <= edges[d + 1]))[0]
            sample += [int(i) for i in idx[np.linspace(0, len(idx) - 1, min(per_cell, len(idx))).astype(int)]]
    return sorted(set(sample))


def test_uneven_batch_full_size(ctx, tcm):
    """4,096 uneven pairs (N log-uniform in [100, 1e5], L in {8, 12, 16, 24}) in one batched call."""
    from paper_0704_1672_gb300 import autotune
    b = synth.uneven_batch()
    T = [(torch.tensor(s, dtype=torch.float32, device="cuda"), None, None) for s in b.systems]
    pb = tcm.pack_batch(T, b.pair_a, b.pair_b, b.L, b.R0, rotB=b.rotB)
    t_default = autotune.moment_phase_ms(ctx, lambda: ctx.tcm_energy_batch_packed(pb, tcm.TCM_MIXED), 3)
    # autotuned tiling (per degree, on a sample of the batch's own items), then the full batch
    res = autotune.tune(ctx, T, b.pair_a, b.pair_b, b.L, b.R0, rotB=b.rotB, precision=tcm.TCM_MIXED,
                        reps=2, max_items_per_l=256)
    t_tuned = autotune.moment_phase_ms(ctx, lambda: ctx.tcm_energy_batch_packed(pb, tcm.TCM_MIXED), 3)
    print(f"moment phase of the full batch: default tiling {t_default:.3f} ms, tuned {t_tuned:.3f} ms; "
          f"choice per L {res.best}")
    E, st = ctx.tcm_energy_batch_packed(pb, tcm.TCM_MIXED)
    torch.cuda.synchronize()
    assert torch.all(st == tcm.TCM_OK)
    E = E.cpu().numpy()
    assert np.all(np.isfinite(E))
    n = np.array([len(s) for s in b.systems])
    sizes = n[b.pair_a] + n[b.pair_b]
    # sample: every degree in every size decile, plus the smallest and largest pair of each degree
    sample = uneven_sample(b)
    for L in (8, 12, 16, 24):
        idx = np.where(b.L == L)[0]
        sample += [int(idx[np.argmin(sizes[idx])]), int(idx[np.argmax(sizes[idx])])]
    sample = sorted(set(sample))
    assert len(sample) >= 64
    check_items("uneven batch", lambda k: b.systems[b.pair_a[k]], lambda k: b.systems[b.pair_b[k]], b.rotB, b.R0,
                b.L, E, sample)
    # the same items alone give bit-identical energies
    for k in sample[::16]:
        E1, _ = ctx.tcm_energy_batch(T, [b.pair_a[k]], [b.pair_b[k]], [b.L[k]], b.R0[k:k + 1], rotB=b.rotB[k:k + 1],
                                     precision=tcm.TCM_MIXED)
        torch.cuda.synchronize()
        assert float(E1[0]) == E[k]
    for L in res.best:  # later tests in this module run with the default tiling and chunking
        ctx.tcm_ctx_set_tiling_l(tcm.TCM_MIXED, L, 64, 2)
        ctx.tcm_ctx_set_chunking_l(L, 160)


def test_large_assembly_full_size(ctx, tcm):
    """1e6-charge shell against a 5e4-atom ligand, 10,000 orientations at Lmax = 24, B's moments
    recomputed per orientation."""
    a = synth.large_assembly()
    A = torch.tensor(a.A, dtype=torch.float32, device="cuda")
    B = torch.tensor(a.B, dtype=torch.float32, device="cuda")
    k = len(a.R0)
    E, st = ctx.tcm_energy_batch([(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int),
                                 np.full(k, a.L), a.R0, rotB=a.rotB, precision=tcm.TCM_MIXED)
    torch.cuda.synchronize()
    assert torch.all(st == tcm.TCM_OK)
    E = E.cpu().numpy()
    L = np.full(k, a.L)
    Af, Bf = f32(a.A), f32(a.B)
    cA, _ = oracle.center_radius(Af)
    cB, _ = oracle.center_radius(Bf)
    QA = oracle_moments_threaded(Af, cA, a.L)
    rep = MixedEnergyReport("large assembly, 16 of 10,000 orientations")
    for kk in np.unique(np.concatenate([np.linspace(0, k - 1, 16).astype(int), [4321]])):
        QB = oracle_moments_threaded(Bf, cB, a.L, rot=a.rotB[kk])
        rep.add(float(E[kk]), oracle.tcm_energy(a.L, QA, QB, a.R0[kk]), oracle.tcm_blocks(a.L, QA, QB, a.R0[kk]),
                f"orientation {kk}")
    assert len(rep.rows) >= 16
    rep.check()


def test_uneven_batch_fp64_subset(ctx, tcm):
    """The double path through the same batched call on a slice of the uneven workload."""
    b = synth.uneven_batch(n_pairs=64, seed=31)
    T = [(torch.tensor(s, dtype=torch.float64, device="cuda"), None, None) for s in b.systems]
    E, st = ctx.tcm_energy_batch(T, b.pair_a, b.pair_b, b.L, b.R0, rotB=b.rotB, precision=tcm.TCM_FP64)
    torch.cuda.synchronize()
    assert torch.all(st == tcm.TCM_OK)
    E = E.cpu().numpy()
    worst = 0.0
    for k in range(0, 64, 9):
        A, B = b.systems[b.pair_a[k]], b.systems[b.pair_b[k]]
        cA, _ = oracle.center_radius(A)
        cB, _ = oracle.center_radius(B)
        QA = oracle_moments_threaded(A, cA, b.L[k])
        QB = oracle_moments_threaded(B, cB, b.L[k], rot=b.rotB[k])
        Eo = oracle.tcm_energy(b.L[k], QA, QB, b.R0[k])
        worst = max(worst, energy_error(float(E[k]), Eo, oracle.tcm_blocks(b.L[k], QA, QB, b.R0[k])))
    assert worst < TOL_FP64, worst
