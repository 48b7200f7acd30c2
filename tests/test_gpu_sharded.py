"""The sharded moment route through the library on one GPU: one system split into atom shards,
each shard's coordinate sums, radius about the global centre and moments about it computed by
libtcm.so (tcm_prepare, tcm_moments), the shards' results combined as the all-reduces of
parallel.sharded_moments combine them (a sum of the coordinate sums, a max of the radii, a sum of
the packed moments: Eq. (multipole) is a sum over atoms), and the result compared with the
oracle's moments of the whole system."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import parallel, synth
from tcm_testlib import TOL_FP64, TOL_MIX_MOM, degree_scales, moment_error, oracle_moments_threaded

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


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision_name", ["TCM_FP64", "TCM_MIXED"])
def test_sharded_moments_through_the_library(tcm, world, precision_name):
    precision = getattr(tcm, precision_name)
    rng = np.random.default_rng(40 + world)
    n = 45001
    S = synth.pack(synth.random_walk(rng, n, 1.9 * n ** (1 / 3)) + [12.0, -7.0, 3.0],
                   synth.charges_normal_net_zero(rng, n))
    dt = torch.float64 if precision == tcm.TCM_FP64 else torch.float32
    Sx = S if precision == tcm.TCM_FP64 else S.astype(np.float32).astype(np.float64)
    L = 16
    shards = []
    for r in range(world):
        lo, hi = parallel.shard_range(n, r, world)
        shards.append(torch.tensor(Sx[lo:hi], dtype=dt, device="cuda"))
    with tcm.Context(lmax_cap=24) as ctx:
        s = sum(parallel.shard_center_sums(ctx, x) for x in shards)        # the sum-all-reduce
        c = s[:3] / s[3]
        a = max(parallel.shard_radius(ctx, x, c) for x in shards)          # the max-all-reduce
        q = sum(parallel.shard_moments(ctx, x, L, c, a, precision) for x in shards)  # the moment all-reduce
        whole = ctx.tcm_moments(torch.tensor(Sx, dtype=dt, device="cuda"), L, precision=precision)
    c_ref, a_ref = oracle.center_radius(Sx)
    assert np.allclose(c, c_ref, rtol=0, atol=1e-12 * 20) and abs(a - a_ref) <= 1e-12 * a_ref, (c, c_ref, a, a_ref)
    sc = degree_scales(Sx, c_ref, L)
    Q = oracle_moments_threaded(Sx, c_ref, L)
    tol = TOL_FP64 if precision == tcm.TCM_FP64 else TOL_MIX_MOM
    err = moment_error(tcm.unpack(q), Q, sc)
    print(f"{world} shards, {precision_name}: moment error {err:.2e} against the oracle")
    assert err < tol
    assert moment_error(tcm.unpack(whole.q), Q, sc) < tol
