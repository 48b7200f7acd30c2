"""The mixed path's L-chunking: the float moment kernel is built for two accumulator budgets
(160 and 96 per lane; tcm_ctx_set_chunking_l chooses one per degree).  Moments of every degree
under the small budget against the oracle at the mixed tolerance, a batch whose degrees use both
budgets (one moment launch per budget) against the oracle, and the setter's checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
from tcm_testlib import TOL_MIX_MOM, MixedEnergyReport, degree_scales, moment_error, oracle_moments_threaded

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


def system(seed, n, radius, shift=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    S = synth.pack(synth.random_walk(rng, n, radius), synth.charges_normal_net_zero(rng, n))
    S[:, :3] += shift
    return S.astype(np.float32).astype(np.float64)


def test_chunking_setter(tcm):
    with tcm.Context(lmax_cap=24) as ctx:
        assert ctx.tcm_ctx_get_chunking_l(24) == (160, 5)
        ctx.tcm_ctx_set_chunking_l(24, 96)
        km, nch = ctx.tcm_ctx_get_chunking_l(24)
        assert (km, nch) == (96, 8)
        assert ctx.tcm_ctx_get_chunking_l(8) == (160, 1)
        for bad in ((24, 128), (25, 160), (-1, 96)):
            with pytest.raises(tcm.TcmError) as e:
                ctx.tcm_ctx_set_chunking_l(*bad)
            assert e.value.code == tcm.TCM_EINVAL
        ctx.tcm_ctx_set_tiling_l(tcm.TCM_MIXED, 24, 64, 3)
        with pytest.raises(tcm.TcmError):
            ctx.tcm_ctx_set_tiling_l(tcm.TCM_FP64, 24, 64, 3)


@pytest.mark.parametrize("L", [0, 3, 8, 9, 12, 13, 16, 20, 24])
def test_small_budget_moments_vs_oracle(tcm, L):
    S = system(40 + L, 9000, 25.0, shift=(5.0, -3.0, 1.0))
    rot = synth.random_rotations(np.random.default_rng(L), 1)[0]
    with tcm.Context(lmax_cap=24) as ctx:
        ctx.tcm_ctx_set_chunking_l(L, 96)
        ctx.tcm_ctx_set_tiling_l(tcm.TCM_MIXED, L, 32, 3)
        m = ctx.tcm_moments(torch.tensor(S, dtype=torch.float32, device="cuda"), L, precision=tcm.TCM_MIXED, rot=rot)
        ctx.tcm_ctx_set_chunking_l(L, 160)
        m160 = ctx.tcm_moments(torch.tensor(S, dtype=torch.float32, device="cuda"), L, precision=tcm.TCM_MIXED,
                               rot=rot)
        torch.cuda.synchronize()
    ref = oracle_moments_threaded(S, m.center, L, rot=rot)
    sc = degree_scales(S, m.center, L, rot=rot)
    err = moment_error(tcm.unpack(m.q), ref, sc)
    assert err < TOL_MIX_MOM, err
    assert moment_error(tcm.unpack(m160.q), ref, sc) < TOL_MIX_MOM


def test_batch_with_both_budgets(tcm):
    rng = np.random.default_rng(12)
    sys_np = [system(60 + i, n, 1.9 * n ** (1 / 3)) for i, n in enumerate((700, 5000, 21000))]
    rad = [oracle.center_radius(S)[1] for S in sys_np]
    T = [(torch.tensor(S, dtype=torch.float32, device="cuda"), None, None) for S in sys_np]
    k = 60
    a, b = rng.integers(0, 3, k), rng.integers(0, 3, k)
    L = rng.choice([6, 10, 16, 24], k)
    R0 = np.array([synth.unit_vectors(rng, 1)[0] * rng.uniform(1.2, 3.0) * (rad[i] + rad[j]) for i, j in zip(a, b)])
    rot = synth.random_rotations(rng, k)
    with tcm.Context(lmax_cap=24) as ctx:
        ctx.tcm_ctx_set_chunking_l(10, 96)
        ctx.tcm_ctx_set_chunking_l(24, 96)
        ctx.tcm_ctx_set_tiling_l(tcm.TCM_MIXED, 24, 64, 3)
        ctx.tcm_ctx_set_profiling(True)
        ctx.tcm_ctx_read_profile()
        E, st = ctx.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=tcm.TCM_MIXED)
        _, launches = ctx.tcm_ctx_read_profile()
        torch.cuda.synchronize()
        assert bool(torch.all(st == 0))
        assert launches["moments"] == 2  # one launch per chunk budget
        E = E.cpu().numpy()
    rep = MixedEnergyReport("batch with both chunk budgets")
    for i in range(0, k, 3):
        A, B = sys_np[a[i]], sys_np[b[i]]
        cA, cB = oracle.center_radius(A)[0], oracle.center_radius(B)[0]
        QA = oracle_moments_threaded(A, cA, int(L[i]))
        QB = oracle_moments_threaded(B, cB, int(L[i]), rot=rot[i])
        rep.add(float(E[i]), oracle.tcm_energy(int(L[i]), QA, QB, R0[i]), oracle.tcm_blocks(int(L[i]), QA, QB, R0[i]),
                f"item {i} (L={L[i]})")
    rep.check()
