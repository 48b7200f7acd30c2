"""The autotuner's host logic on CPU: degree grouping, the sweep over candidates, choosing and
applying the fastest, and the JSON cache, with a fake context whose 'time' is a known function
of the tiling (no GPU).  The GPU test tunes a real uneven batch and checks the results still
match the oracle."""
import numpy as np
import pytest

from paper_0704_1672_gb300 import autotune, synth, tcm


class FakeCtx:
    def __init__(self):
        self.tiling = {}
        self.chunking = {}
        self.calls = 0

    def tcm_ctx_get_tiling_l(self, precision, L):
        return self.tiling.get((precision, L), (64, 2))

    def tcm_ctx_set_tiling_l(self, precision, L, apl, cps):
        assert 1 <= cps <= (2 if precision == tcm.TCM_FP64 else 3)
        self.tiling[(precision, L)] = (apl, cps)

    def tcm_ctx_get_chunking_l(self, L):
        k = self.chunking.get(L, 160)
        return k, -(-(L + 1) ** 2 // k)

    def tcm_ctx_set_chunking_l(self, L, kmax):
        assert kmax in (160, 96)
        self.chunking[L] = kmax

    def setting(self, precision, L):
        apl, cps = self.tcm_ctx_get_tiling_l(precision, L)
        return (apl, cps, self.chunking.get(L, 160) if precision != tcm.TCM_FP64 else 80)

    def tcm_energy_batch_packed(self, pb, precision, E=None, status=None):
        self.calls += 1


def cost(L, apl, cps, kmax):
    # a made-up landscape with its minimum at apl = 2**(3 + L // 8), cps = 1 for odd L, and the
    # small chunk budget (kmax 96, with 3 CTAs per SM) for L < 16
    c = abs(np.log2(apl) - (3 + L // 8)) + (0.5 if (cps == 1) != (L % 2 == 1) else 0.0) + 0.01 * L
    if L < 16:
        c += 0.0 if (kmax == 96 and cps == 3) else 1.0
    else:
        c += 0.0 if kmax == 160 else 0.7
    return c


def systems(n):
    return [tcm.tcm_system() for _ in range(n)]


def test_degree_groups_cap_and_cover():
    lmax = np.array([8, 12, 8, 24, 8, 12, 8])
    g = autotune.degree_groups(lmax, 2)
    assert sorted(g) == [8, 12, 24]
    assert list(g[12]) == [1, 5] and list(g[24]) == [3]
    assert len(g[8]) == 2 and set(g[8]) <= {0, 2, 4, 6} and g[8][0] == 0 and g[8][-1] == 6


def test_tune_picks_the_fastest_per_degree_and_applies_it():
    ctx = FakeCtx()
    rng = np.random.default_rng(0)
    k = 40
    L = rng.choice([8, 13, 16, 24], k)
    R0 = rng.normal(size=(k, 3)) + 50.0

    def measure(Ldeg, run):
        run()
        return cost(Ldeg, *ctx.setting(tcm.TCM_MIXED, Ldeg))

    res = autotune.tune(ctx, systems(3), rng.integers(0, 3, k), rng.integers(0, 3, k), L, R0,
                        rotB=synth.random_rotations(rng, k), precision=tcm.TCM_MIXED, measure=measure)
    # the candidates: every atoms-per-lane value with CTAs per SM up to what each budget's kernel
    # is compiled for (2 at kmax 160, 3 at kmax 96)
    grid = {(a, c, km): cost(0, a, c, km) for km in (160, 96) for a in autotune.DEFAULT_ATOMS_PER_LANE
            for c in (1, 2, 3) if c <= (2 if km == 160 else 3)}
    assert len(autotune.candidates(tcm.TCM_MIXED)) == len(grid) == 5 * len(autotune.DEFAULT_ATOMS_PER_LANE)
    for Ldeg in (8, 13, 16, 24):
        grid = {cand: cost(Ldeg, *cand) for cand in autotune.candidates(tcm.TCM_MIXED)}
        want = min(grid, key=grid.get)
        assert res.best[Ldeg] == want
        assert ctx.setting(tcm.TCM_MIXED, Ldeg) == want
        assert res.timings[Ldeg] == pytest.approx(grid)
    assert res.best[8][2] == 96 and res.best[24][2] == 160
    assert ctx.calls == 4 * len(autotune.candidates(tcm.TCM_MIXED))


def test_choose_prefers_larger_tiles_within_one_percent():
    t = {(64, 2, 160): 1.000, (128, 2, 160): 1.005, (256, 2, 160): 1.012, (512, 1, 160): 1.008, (32, 3, 96): 0.999}
    assert autotune.choose(t) == (512, 1, 160)          # 1.008 <= 1.01 * 0.999: the largest tiles within 1 %
    assert autotune.choose(t, tol=0.0) == (32, 3, 96)   # the fastest alone
    assert autotune.choose({}) is None


def test_larger_tiles_preferred_only_when_the_degree_was_sampled():
    def landscape(L, apl, cps, km):
        return {256: 1.000, 512: 1.005}.get(apl, 2.0) + (0.0 if (cps, km) == (2, 160) else 1.0)

    rng = np.random.default_rng(3)
    k = 10
    R0 = rng.normal(size=(k, 3)) + 50.0
    for cap, want in ((4, 512), (512, 256)):  # 4 of the 10 items: a sample; 512: all of them
        ctx = FakeCtx()
        res = autotune.tune(ctx, systems(2), np.zeros(k, int), np.ones(k, int), np.full(k, 24), R0,
                            precision=tcm.TCM_MIXED, max_items_per_l=cap, atoms_per_lane=(64, 256, 512),
                            measure=lambda L, run: (run(), landscape(L, *ctx.setting(tcm.TCM_MIXED, L)))[1])
        assert res.best[24] == (want, 2, 160), (cap, res.best)


def test_fp64_candidates_keep_the_double_budget():
    c = autotune.candidates(tcm.TCM_FP64, (32, 64), (1, 2, 3))
    assert c == [(32, 1, 80), (32, 2, 80), (64, 1, 80), (64, 2, 80)]


def test_cache_round_trip(tmp_path):
    ctx = FakeCtx()
    r = autotune.TuneResult(tcm.TCM_MIXED, best={8: (32, 3, 96), 24: (128, 2, 160)},
                            timings={8: {(32, 3, 96): 0.1, (64, 2, 160): 0.2}, 24: {(128, 2, 160): 0.3}})
    path = str(tmp_path / "tiling.json")
    autotune.save(path, r, "GB300|abc")
    autotune.save(path, autotune.TuneResult(tcm.TCM_FP64, best={8: (16, 2, 80)}), "GB300|abc")
    assert autotune.load(ctx, path, tcm.TCM_MIXED, "other|key") is None
    got = autotune.load(ctx, path, tcm.TCM_MIXED, "GB300|abc")
    assert got.best == r.best and got.timings == r.timings
    assert ctx.tiling == {(tcm.TCM_MIXED, 8): (32, 3), (tcm.TCM_MIXED, 24): (128, 2)}
    assert ctx.chunking == {8: 96, 24: 160}
    assert autotune.load(ctx, path, tcm.TCM_FP64, "GB300|abc").best == {8: (16, 2, 80)}


@pytest.mark.gpu
def test_tuned_uneven_batch_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_0704_1672_gb300 import build
    build.build()
    from tcm_testlib import MixedEnergyReport, oracle_moments_threaded
    rng = np.random.default_rng(31)
    sizes = [150, 900, 4000, 15000, 30000]
    sys_np, T, rad = [], [], []
    for n in sizes:
        xyz = synth.random_walk(rng, n, 1.9 * n ** (1 / 3))
        S = synth.pack(xyz, synth.charges_normal_net_zero(rng, n))
        sys_np.append(S)
        T.append((torch.tensor(S, dtype=torch.float32, device="cuda"), None, None))
        rad.append(oracle.center_radius(S.astype(np.float32).astype(np.float64))[1])
    k = 48
    a = rng.integers(0, len(sizes), k)
    b = rng.integers(0, len(sizes), k)
    L = rng.choice([8, 12, 16, 24], k)
    R0 = np.array([synth.unit_vectors(rng, 1)[0] * rng.uniform(1.2, 3.0) * (rad[i] + rad[j]) for i, j in zip(a, b)])
    rot = synth.random_rotations(rng, k)
    ctx = tcm.Context(lmax_cap=24)
    try:
        res = autotune.tune(ctx, T, a, b, L, R0, rotB=rot, reps=2)
        assert sorted(res.best) == [8, 12, 16, 24]
        for Ldeg, best in res.best.items():
            assert autotune.get_setting(ctx, tcm.TCM_MIXED, Ldeg) == best
            assert res.timings[Ldeg][best] <= 1.01 * min(res.timings[Ldeg].values())
        print({Ldeg: (best, round(res.timings[Ldeg][best], 4)) for Ldeg, best in res.best.items()})
        E, st = ctx.tcm_energy_batch(T, a, b, L, R0, rotB=rot)
        torch.cuda.synchronize()
        assert bool(torch.all(st == 0))
        rep = MixedEnergyReport("tuned uneven batch")
        for i in range(0, k, 7):
            A = sys_np[a[i]].astype(np.float32).astype(np.float64)
            B = sys_np[b[i]].astype(np.float32).astype(np.float64)
            cA, cB = oracle.center_radius(A)[0], oracle.center_radius(B)[0]
            QA = oracle_moments_threaded(A, cA, int(L[i]))
            QB = oracle_moments_threaded(B, cB, int(L[i]), rot=rot[i])
            rep.add(float(E[i]), oracle.tcm_energy(int(L[i]), QA, QB, R0[i]),
                    oracle.tcm_blocks(int(L[i]), QA, QB, R0[i]), f"item {i}")
        rep.check()
    finally:
        ctx.close()
