"""The serving engine: scheduling and admission on CPU with a fake executor (faults made on the
host), and the GPU executor's results against the same requests served alone and the oracle."""
import numpy as np
import pytest

from paper_0704_1672_gb300 import synth
from paper_0704_1672_gb300.serve import Engine, Request


class FakeExecutor:
    """Deterministic stand-in for the GPU: an item's 'energy' depends only on the item; a batch
    becomes ready after `latency` polls; items with R0 = 0 come back with status 2 (not converged)."""

    def __init__(self, latency=2):
        self.latency = latency
        self.batches = []

    def submit(self, batch):
        E = np.array([a * 1000 + b * 10 + L + float(np.sum(R)) for a, b, L, R in zip(batch.a, batch.b, batch.L, batch.R0)])
        st = np.array([2 if not np.any(R) else 0 for R in batch.R0], dtype=np.int32)
        h = {"polls": 0, "E": E, "st": st, "n": len(batch)}
        self.batches.append(h)
        return h

    def ready(self, h):
        h["polls"] += 1
        return h["polls"] > self.latency

    def wait(self, h):
        h["polls"] = self.latency + 1

    def collect(self, h):
        return h["E"], h["st"]


def req(rid, n, a=0, b=1, L=4, seed=0):
    rng = np.random.default_rng(seed + rid)
    return Request(rid, a, b, L, synth.random_rotations(rng, n), rng.normal(size=(n, 3)) + 10.0)


def expected(r):
    return np.array([r.a * 1000 + r.b * 10 + r.L + float(np.sum(R)) for R in r.R0])


def test_all_requests_served_and_results_match_alone():
    ex = FakeExecutor()
    eng = Engine(ex, lambda r: 100, budget_bytes=10 ** 9, max_items=64, quota=16)
    rs = [req(i, n, a=i % 5, b=(i + 1) % 5, L=4 + i % 3) for i, n in enumerate([1, 40, 7, 200, 3, 64])]
    for r in rs:
        eng.submit(r)
    eng.drain()
    assert [r.state for r in rs] == ["done"] * len(rs)
    for r in rs:
        assert np.array_equal(r.E, expected(r)) and np.all(r.status == 0)
    assert any(len(h["E"]) > 16 for h in ex.batches)


def test_admission_by_budget_and_rejection():
    ex = FakeExecutor()
    eng = Engine(ex, lambda r: 1000, budget_bytes=20_000, max_items=8, quota=8)
    big = req(0, 100)     # footprint 8 items x 1000 = 8000
    huge = req(1, 100)
    never = req(2, 100)
    eng.item_bytes = lambda r: 3000 if r.rid == 2 else 1000  # 8 x 3000 = 24000 > budget: rejected
    assert eng.submit(big)
    assert eng.submit(huge)
    assert not eng.submit(never)
    assert never.state == "rejected"
    eng.step()
    assert eng.used <= eng.budget
    eng.drain()
    assert big.state == huge.state == "done"
    assert eng.used == 0


def test_budget_holds_back_requests_until_memory_frees():
    ex = FakeExecutor(latency=1)
    eng = Engine(ex, lambda r: 1000, budget_bytes=8000, max_items=8, quota=8)
    a, b = req(0, 16), req(1, 16)
    eng.submit(a)
    eng.submit(b)
    eng.step()
    assert a.state == "active" and b.state == "pending"  # b waits for a's memory
    eng.drain()
    assert a.state == b.state == "done"
    assert b.t_admit >= a.t_done


def test_long_scan_does_not_starve_short_requests():
    ex = FakeExecutor(latency=1)
    eng = Engine(ex, lambda r: 10, budget_bytes=10 ** 9, max_items=32, quota=8)
    long = req(0, 2000)
    eng.submit(long)
    for _ in range(3):
        eng.step()
    shorts = [req(i, 4) for i in range(1, 6)]
    for r in shorts:
        eng.submit(r)
    eng.drain()
    assert all(r.t_done < long.t_done for r in shorts)


def test_cancel_mid_scan_discards_in_flight_results():
    ex = FakeExecutor(latency=3)
    eng = Engine(ex, lambda r: 10, budget_bytes=10 ** 9, max_items=16, quota=16)
    a, b = req(0, 100), req(1, 10)
    eng.submit(a)
    eng.submit(b)
    eng.step()  # a's first items are in flight
    eng.cancel(a)
    eng.drain()
    assert a.state == "cancelled" and a.done_items < a.n
    assert b.state == "done" and np.array_equal(b.E, expected(b))
    assert eng.used == 0


def test_not_converged_items_report_status():
    ex = FakeExecutor()
    eng = Engine(ex, lambda r: 10)
    r = req(0, 5)
    r.R0[2] = 0.0
    eng.submit(r)
    eng.drain()
    assert r.state == "done" and list(r.status) == [0, 0, 2, 0, 0]


@pytest.mark.gpu
@pytest.mark.parametrize("rotate_cached", [False, True])
def test_gpu_engine_results_same_alone_and_in_mix(rotate_cached):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_0704_1672_gb300 import build
    build.build()
    from paper_0704_1672_gb300.serve import GpuExecutor, make_requests
    from tcm_testlib import MixedEnergyReport, oracle_moments_threaded

    st = synth.serve_stream(seed=9, n_pool=12, n_lo=300, n_hi=6000, rate=4000.0, seconds=0.05, orient_hi=24)
    ex = GpuExecutor(st.systems, lmax_cap=24, rotate_cached=rotate_cached)
    reqs = make_requests(st)
    eng = Engine(ex, ex.item_bytes, max_items=256, quota=32)
    m = eng.run_stream(reqs)
    assert m["requests_done"] == len(reqs) and m["latency_ms"]["p99"] is not None
    done = {r.rid: r for r in eng.done}
    sample = [reqs[0].rid, reqs[len(reqs) // 2].rid, reqs[-1].rid]
    for rid in sample:
        r = done[rid]
        alone = Request(rid, r.a, r.b, r.L, r.rot, r.R0)
        eng2 = Engine(ex, ex.item_bytes, max_items=256, quota=32)
        eng2.submit(alone)
        eng2.drain()
        assert np.array_equal(alone.E, r.E), (rid, alone.E - r.E)
    # and the served energies are right
    r = done[sample[0]]
    A = st.systems[r.a].astype(np.float32).astype(np.float64)
    B = st.systems[r.b].astype(np.float32).astype(np.float64)
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    QA = oracle_moments_threaded(A, cA, r.L)
    rep = MixedEnergyReport("served request")
    for k in range(min(3, r.n)):
        QB = oracle_moments_threaded(B, cB, r.L, rot=r.rot[k])
        rep.add(r.E[k], oracle.tcm_energy(r.L, QA, QB, r.R0[k]), oracle.tcm_blocks(r.L, QA, QB, r.R0[k]), f"item {k}")
    rep.check()
