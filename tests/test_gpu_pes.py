"""The surface scan of Section IV at full size (15,480 grid points, Lmax in {1, 2, 3, 4, 6, 8,
10}, exact energies at every point): sampled grid points against the oracle's Eq. (Formula) and
Eq. (Coulomb), and the relative error of Eq. (error) falling with Lmax."""
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


@pytest.mark.parametrize("precision_name,dr,dtheta", [("TCM_MIXED", 1.0, 1.0), ("TCM_FP64", 6.0, 30.0)])
def test_surface_scan(tcm, precision_name, dr, dtheta):
    from paper_0704_1672_gb300 import pes
    precision = getattr(tcm, precision_name)
    g = synth.pes_grid_pair(dr=dr, dtheta=dtheta)
    A = torch.tensor(g.A, device="cuda")
    B = torch.tensor(g.B, device="cuda")
    R0 = g.R0()
    ctx = tcm.Context(lmax_cap=24)
    try:
        res = pes.scan(ctx, A, B, R0, g.lmax, precision=precision)
    finally:
        ctx.close()
    n = len(R0)
    print(f"{n} grid points: {res.timings_ms}")
    cA, aA = oracle.center_radius(g.A)
    cB, aB = oracle.center_radius(g.B)
    assert np.allclose(res.centers[0], cA, atol=1e-12) and np.allclose(res.centers[1], cB, atol=1e-12)
    Lhi = max(g.lmax)
    QA = oracle_moments_threaded(g.A, cA, Lhi)
    QB = oracle_moments_threaded(g.B, cB, Lhi)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 6)]))
    rep = MixedEnergyReport("surface scan")
    for i in sample:
        Ed, sc = oracle.direct(g.A, cA, g.B, cB, R0[i], return_abs=True)
        assert abs(res.U_coul[i] - Ed) < 1e-12 * sc, (i, res.U_coul[i], Ed)
        for L in g.lmax:
            Eo = oracle.tcm_energy(L, QA, QB, R0[i])
            blocks = oracle.tcm_blocks(L, QA, QB, R0[i])
            if precision == tcm.TCM_MIXED:
                rep.add(res.U_mult[L][i], Eo, blocks, f"point {i}, Lmax {L}")
            else:
                assert energy_error(res.U_mult[L][i], Eo, blocks) < TOL_FP64, (i, L)
    if precision == tcm.TCM_MIXED:
        rep.check()
    med = [float(np.median(res.eta(L))) for L in g.lmax]
    mx = [float(np.max(res.eta(L))) for L in g.lmax]
    print("Eq. (error) median / max per Lmax (%):",
          {L: (round(m, 4), round(x, 4)) for L, m, x in zip(g.lmax, med, mx)})
    assert all(b < a for a, b in zip(med, med[1:])), med
