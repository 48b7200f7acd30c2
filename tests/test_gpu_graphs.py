"""CUDA-graph replay of the batched call: a replayed launch sequence gives bit-identical results to
kernel-by-kernel launches on the same inputs, reads each call's new descriptors (new orientations,
same shapes), and is captured again when the launch shapes change."""
import numpy as np
import pytest
import torch

from paper_0704_1672_gb300 import synth

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


def _systems():
    out = []
    for i, (n, r) in enumerate([(700, 6.0), (5000, 10.0), (20000, 16.0)]):
        rng = np.random.default_rng(500 + i)
        S = synth.pack(synth.uniform_ball(rng, n, r), synth.charges_uniform_net_zero(rng, n))
        out.append(torch.tensor(S, dtype=torch.float32, device="cuda"))
    return out


def _items(seed, k, rad):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 3, k)
    b = rng.integers(0, 3, k)
    L = rng.integers(4, 21, k)
    R0 = np.array([synth.unit_vectors(rng, 1)[0] * 1.6 * (rad[i] + rad[j]) for i, j in zip(a, b)])
    return a, b, L, R0, synth.random_rotations(rng, k)


@pytest.mark.parametrize("precision_name", ["TCM_MIXED", "TCM_FP64"])
def test_graph_replay_matches_direct_launches(tcm, precision_name):
    precision = getattr(tcm, precision_name)
    T = [(s, None, None) for s in _systems()]
    rad = [6.0, 10.0, 16.0]
    k = 96
    E = torch.empty(k, dtype=torch.float64, device="cuda")
    st = torch.empty(k, dtype=torch.int32, device="cuda")
    direct = tcm.Context(lmax_cap=24)
    direct.tcm_ctx_set_graphs(False)
    graph = tcm.Context(lmax_cap=24)
    try:
        for rep, seed in enumerate([1, 1, 2, 3]):
            a, b, L, R0, rot = _items(seed, k, rad)
            # same item shapes (L per slot) in every call: only orientations and pairs vary
            L = _items(1, k, rad)[2]
            Ed, sd = direct.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision)
            graph.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision, E=E, status=st)
            torch.cuda.synchronize()
            assert torch.equal(Ed, E), (rep, (Ed - E).abs().max().item())
            assert torch.equal(sd, st)
        cap, lau = graph.tcm_ctx_graph_stats()
        assert cap >= 1 and lau >= 1  # the repeated first call was captured and replayed
        assert direct.tcm_ctx_graph_stats() == (0, 0)
        # same shape, new orientations: replays of the captured graph read the new descriptors
        a, b, L, R0, rot = _items(1, k, rad)
        for rep in range(3):
            R0 = R0 * (1.0 + 0.05 * rep)
            rot = np.ascontiguousarray(np.roll(rot, rep, axis=0))
            Ed, _ = direct.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision)
            graph.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision, E=E, status=st)
            torch.cuda.synchronize()
            assert torch.equal(Ed, E), rep
        cap2, lau2 = graph.tcm_ctx_graph_stats()
        assert lau2 >= lau + 2 and cap2 <= cap + 1
        # a different batch size: launched directly once, captured on its repeat
        a, b, L, R0, rot = _items(7, 33, rad)
        E2 = torch.empty(33, dtype=torch.float64, device="cuda")
        s2 = torch.empty(33, dtype=torch.int32, device="cuda")
        for rep in range(2):
            graph.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision, E=E2, status=s2)
            Ed, _ = direct.tcm_energy_batch(T, a, b, L, R0, rotB=rot, precision=precision)
            torch.cuda.synchronize()
            assert torch.equal(Ed, E2)
        assert graph.tcm_ctx_graph_stats() == (cap2 + 1, lau2 + 1)
    finally:
        direct.close()
        graph.close()


def test_graph_replay_with_cached_moments(tcm):
    """The serving path (moments cached in the system descriptors) replays too."""
    sys_t = _systems()
    ctx = tcm.Context(lmax_cap=24)
    ref = tcm.Context(lmax_cap=24)
    ref.tcm_ctx_set_graphs(False)
    try:
        cached, keep = [], []
        for s in sys_t:
            m = ctx.tcm_moments(s, 24, precision=tcm.TCM_MIXED)
            keep.append(m)
            cached.append(tcm.make_system(s, m.center, m.radius, moments=m))
        rad = [6.0, 10.0, 16.0]
        k = 64
        E = torch.empty(k, dtype=torch.float64, device="cuda")
        st = torch.empty(k, dtype=torch.int32, device="cuda")
        a, b, L, R0, rot = _items(3, k, rad)
        for rep in range(4):
            R0 = R0 * (1.0 + 0.05 * rep)
            rot = np.ascontiguousarray(np.roll(rot, rep, axis=0))
            ctx.tcm_energy_batch(cached, a, b, L, R0, rotB=rot, E=E, status=st)
            Ed, _ = ref.tcm_energy_batch(cached, a, b, L, R0, rotB=rot)
            torch.cuda.synchronize()
            assert torch.equal(Ed, E)
        assert ctx.tcm_ctx_graph_stats()[1] >= 2
    finally:
        ctx.close()
        ref.close()


def test_graph_replay_of_gradients(tcm):
    """The gradient variant of the batched call replays too, with the same forces and torques."""
    T = [(s, None, None) for s in _systems()]
    rad = [6.0, 10.0, 16.0]
    k = 40
    a, b, L, R0, rot = _items(11, k, rad)
    E = torch.empty(k, dtype=torch.float64, device="cuda")
    G = torch.empty((k, 9), dtype=torch.float64, device="cuda")
    st = torch.empty(k, dtype=torch.int32, device="cuda")
    direct = tcm.Context(lmax_cap=24)
    direct.tcm_ctx_set_graphs(False)
    graph = tcm.Context(lmax_cap=24)
    try:
        for rep in range(3):
            R = R0 * (1.0 + 0.03 * rep)
            Ed, Gd, _ = direct.tcm_gradients_batch(T, a, b, L, R, rotB=rot)
            graph.tcm_gradients_batch(T, a, b, L, R, rotB=rot, E=E, G=G, status=st)
            torch.cuda.synchronize()
            assert torch.equal(Ed, E) and torch.equal(Gd, G), rep
        assert graph.tcm_ctx_graph_stats()[1] >= 1
    finally:
        direct.close()
        graph.close()
