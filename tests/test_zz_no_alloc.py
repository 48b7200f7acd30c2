"""tcm_moments_noalloc, the entry point for callers that cannot allocate device memory
(for example code that must not let cudaMalloc/cudaFree synchronise the device, or an
application whose own allocator owns all device memory).  It keeps its scratch in a fixed
array inside the library, so these tests check, through the C ABI, that calls in a row each
give what the allocating entry point tcm_moments gives and what the CPU oracle gives, within
the parity tolerances, that a call leaves nothing behind that changes the next one, and that
the paths its fixed array is dimensioned for (the tiled centre/radius kernels, the largest
atom count, Lmax 24 in double precision) stay inside it.

The file is named to be collected last."""
import numpy as np
import pytest
import torch

import oracle
from paper_0704_1672_gb300 import synth
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


def _system(seed, n, radius, shift):
    rng = np.random.default_rng(seed)
    S = synth.pack(synth.uniform_ball(rng, n, radius), synth.charges_uniform_net_zero(rng, n))
    S[:, :3] += shift
    return S


def _tol(precision, tcm):
    return TOL_FP64 if precision == tcm.TCM_FP64 else TOL_MIX_MOM


def test_noalloc_matches_tcm_moments_and_oracle_on_two_calls_in_a_row(tcm):
    rng = np.random.default_rng(23)
    S1 = _system(1, 9000, 12.0, (4.0, -3.0, 1.0))   # float32 coordinates, mixed, rotated, centre computed
    S2 = _system(2, 5000, 8.0, (-1.0, 2.0, 0.5))    # float64 coordinates, FP64, centre and radius given
    rot = synth.random_rotations(rng, 1)[0]
    c2 = S2[:, :3].mean(0)
    a2 = float(np.sqrt(((S2[:, :3] - c2) ** 2).sum(1)).max())
    A1 = torch.tensor(S1, dtype=torch.float32, device="cuda")
    A2 = torch.tensor(S2, dtype=torch.float64, device="cuda")
    L1, L2 = 20, 24
    with tcm.Context(lmax_cap=24) as ctx:
        ref1 = ctx.tcm_moments(A1, L1, precision=tcm.TCM_MIXED, rot=rot)
        ref2 = ctx.tcm_moments(A2, L2, precision=tcm.TCM_FP64, center=c2, radius=a2)
    out1 = torch.empty((L1 + 1) ** 2, dtype=torch.float64, device="cuda")
    out2 = torch.empty((L2 + 1) ** 2, dtype=torch.float64, device="cuda")
    geo1 = torch.empty(4, dtype=torch.float64, device="cuda")
    geo2 = torch.empty(4, dtype=torch.float64, device="cuda")
    tcm.tcm_moments_noalloc(A1, L1, tcm.TCM_MIXED, rot=rot, out=out1, center_radius_out=geo1)
    tcm.tcm_moments_noalloc(A2, L2, tcm.TCM_FP64, center=c2, radius=a2, out=out2, center_radius_out=geo2)
    torch.cuda.synchronize()
    S1f = S1.astype(np.float32).astype(np.float64)
    c1_ref, a1_ref = oracle.center_radius(S1f)
    g1 = geo1.cpu().numpy()
    assert np.allclose(g1[:3], c1_ref, rtol=0, atol=1e-12) and abs(g1[3] - a1_ref) < 1e-12 * a1_ref
    g2 = geo2.cpu().numpy()
    assert np.array_equal(g2[:3], c2) and g2[3] == a2
    sc1 = degree_scales(S1f, c1_ref, L1, rot=rot)
    sc2 = degree_scales(S2, c2, L2)
    # against the oracle (the independent reference) ...
    Q1 = oracle_moments_threaded(S1f, c1_ref, L1, rot=rot)
    Q2 = oracle_moments_threaded(S2, c2, L2)
    assert moment_error(tcm.unpack(out1), Q1, sc1) < TOL_MIX_MOM
    assert moment_error(tcm.unpack(out2), Q2, sc2) < TOL_FP64
    # ... and against the allocating entry point
    assert moment_error(tcm.unpack(out1), tcm.unpack(ref1.q), sc1) < TOL_MIX_MOM
    assert moment_error(tcm.unpack(out2), tcm.unpack(ref2.q), sc2) < TOL_FP64
    # the shared scratch keeps the previous call's contents; a repeat must not depend on them
    again = torch.empty_like(out1)
    tcm.tcm_moments_noalloc(A1, L1, tcm.TCM_MIXED, rot=rot, out=again)
    torch.cuda.synchronize()
    assert torch.equal(again, out1)


@pytest.mark.parametrize("case", ["float64_centre_computed", "max_atoms_mixed", "max_atoms_fp64"])
def test_noalloc_tiled_centre_and_largest_request(tcm, case):
    """The tiled centre/radius kernels (float64 records, or float32 beyond one thread-block
    cluster) and the largest request the fixed array holds: TCM_NOALLOC_MAX_ATOMS atoms at
    Lmax 24, with the centre and radius computed on the device; two calls in a row."""
    if case == "float64_centre_computed":
        S = _system(5, 20000, 15.0, (30.0, 10.0, -5.0))
        dt, L, precision = torch.float64, 16, tcm.TCM_MIXED
    else:
        S = _system(6, tcm.NOALLOC_MAX_ATOMS, 60.0, (-20.0, 5.0, 40.0))
        dt, L = torch.float32, 24
        precision = tcm.TCM_MIXED if case == "max_atoms_mixed" else tcm.TCM_FP64
    Sx = S.astype(np.float32).astype(np.float64) if dt == torch.float32 else S
    X = torch.tensor(Sx, dtype=dt, device="cuda")
    rot = synth.random_rotations(np.random.default_rng(7), 1)[0]
    with tcm.Context(lmax_cap=24) as ctx:
        ref = ctx.tcm_moments(X, L, precision=precision, rot=rot)
    outs = []
    for _ in range(2):
        out = torch.empty((L + 1) ** 2, dtype=torch.float64, device="cuda")
        geo = torch.empty(4, dtype=torch.float64, device="cuda")
        tcm.tcm_moments_noalloc(X, L, precision, rot=rot, out=out, center_radius_out=geo)
        torch.cuda.synchronize()
        outs.append((out, geo))
    c_ref, a_ref = oracle.center_radius(Sx)
    g = outs[0][1].cpu().numpy()
    assert np.allclose(g[:3], c_ref, rtol=0, atol=1e-11) and abs(g[3] - a_ref) <= 1e-12 * a_ref, (g, c_ref, a_ref)
    sc = degree_scales(Sx, c_ref, L, rot=rot)
    Q = oracle_moments_threaded(Sx, c_ref, L, rot=rot)
    assert moment_error(tcm.unpack(outs[0][0]), Q, sc) < _tol(precision, tcm)
    assert moment_error(tcm.unpack(outs[0][0]), tcm.unpack(ref.q), sc) < _tol(precision, tcm)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_noalloc_rejects_requests_beyond_its_scratch(tcm):
    big = torch.zeros((tcm.NOALLOC_MAX_ATOMS + 1, 4), dtype=torch.float32, device="cuda")
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    with pytest.raises(tcm.TcmError) as e:
        tcm.tcm_moments_noalloc(big, 2, out=out, center=(0, 0, 0), radius=1.0)
    assert e.value.code == tcm.TCM_EINVAL and "262144" in str(e.value)
    small = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(tcm.TcmError) as e:
        tcm.tcm_moments_noalloc(small, 25, out=torch.empty(676, dtype=torch.float64, device="cuda"))
    assert e.value.code == tcm.TCM_EINVAL
    # outputs the call could overrun are refused before anything is queued
    with pytest.raises(tcm.TcmError) as e:
        tcm.tcm_moments_noalloc(small, 4, out=torch.empty(24, dtype=torch.float64, device="cuda"))
    assert e.value.code == tcm.TCM_EINVAL
    with pytest.raises(tcm.TcmError) as e:
        tcm.tcm_moments_noalloc(small, 4, out=torch.empty(25, dtype=torch.float32, device="cuda"))
    assert e.value.code == tcm.TCM_EINVAL
