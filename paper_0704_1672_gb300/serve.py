"""Continuous-batching server for two-center energy / PES-scan requests on one GPU.

A request asks for the energies of one pair (a, b) of resident systems at n orientations of
b (rotation about its centre and separation R0) at one Lmax.  The engine

* keeps every system's coordinates and its moment cache (moments about its centre at the
  pool's Lmax cap, used for the unrotated side a) resident on the device;
* admits requests in arrival order while the device-memory budget and the slot count allow
  (a request that can never fit is rejected at once);
* every iteration packs work items from all active requests into one batched call
  (tcm_energy_batch), at most ``quota`` items per request so that long scans do not starve
  short ones, and queues it on the GPU without waiting; new arrivals join the next
  iteration while earlier ones are still running, so their work overlaps on the device;
* completes a request when its last item comes back and records its latency
  (completion - arrival).

The scheduling logic is independent of the executor; ``GpuExecutor`` drives the C ABI.
"""
from __future__ import annotations

import argparse
import collections
import json
import time
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------- requests

@dataclass(eq=False)  # identity comparison: requests are removed from lists by identity
class Request:
    rid: int
    a: int
    b: int
    L: int
    rot: np.ndarray  # (k, 3, 3)
    R0: np.ndarray  # (k, 3)
    arrival: float = 0.0
    E: np.ndarray = None
    status: np.ndarray = None
    next_item: int = 0
    done_items: int = 0
    t_admit: float = None
    t_done: float = None
    state: str = "pending"  # pending, active, done, rejected, cancelled
    footprint: int = 0

    @property
    def n(self):
        return len(self.R0)


@dataclass
class Batch:
    """Work items of one iteration, as per-request segments (request, first item, count) and the
    items' arrays in slot order."""
    segments: list = field(default_factory=list)
    a: np.ndarray = None
    b: np.ndarray = None
    L: np.ndarray = None
    rot: np.ndarray = None  # (k, 3, 3)
    R0: np.ndarray = None   # (k, 3)

    def __len__(self):
        return 0 if self.a is None else len(self.a)


# ----------------------------------------------------------------------------- engine

class Engine:
    def __init__(self, executor, item_bytes, budget_bytes=4 << 30, max_active=512, max_items=2048, quota=256,
                 depth=2, clock=time.perf_counter):
        """item_bytes(req) -> device bytes one in-flight item of ``req`` needs; budget_bytes bounds the
        sum over active requests of quota-limited footprints."""
        self.ex = executor
        self.item_bytes = item_bytes
        self.budget = budget_bytes
        self.max_active = max_active
        self.max_items = max_items
        self.quota = quota
        self.depth = depth
        self.clock = clock
        self.pending = collections.deque()
        self.active = []
        self.inflight = collections.deque()  # (handle, batch)
        self.used = 0
        self.done = []
        self.rejected = []
        self._rr = 0

    # -- requests
    def submit(self, req: Request):
        req.state = "pending"
        req.E = np.full(req.n, np.nan)
        req.status = np.full(req.n, -1, dtype=np.int32)
        req.footprint = self.item_bytes(req) * min(req.n, self.quota)
        if req.footprint > self.budget or req.n == 0:
            req.state = "rejected"
            req.t_done = self.clock()
            self.rejected.append(req)
            return False
        self.pending.append(req)
        return True

    def cancel(self, req: Request):
        """Drop the request's remaining items; items already on the GPU finish but are discarded."""
        if req.state in ("pending", "active"):
            if req.state == "pending":
                self.pending.remove(req)
            else:
                self.active.remove(req)
                self.used -= req.footprint
            req.state = "cancelled"
            req.t_done = self.clock()

    def _admit(self):
        while self.pending and len(self.active) < self.max_active:
            req = self.pending[0]
            if self.used + req.footprint > self.budget:
                break
            self.pending.popleft()
            req.state = "active"
            req.t_admit = self.clock()
            self.used += req.footprint
            self.active.append(req)

    def _pack(self) -> Batch:
        b = Batch()
        if not self.active:
            return b
        n = len(self.active)
        # round-robin over active requests, at most `quota` items each, up to max_items
        share = max(1, min(self.quota, self.max_items // n))
        order = [self.active[(self._rr + i) % n] for i in range(n)]
        self._rr = (self._rr + 1) % max(1, n)
        total = 0
        for req in order:
            take = min(share, req.n - req.next_item, self.max_items - total)
            if take <= 0:
                continue
            b.segments.append((req, req.next_item, take))
            req.next_item += take
            total += take
            if total >= self.max_items:
                break
        if not b.segments:
            return b
        counts = np.fromiter((t for _, _, t in b.segments), dtype=np.int64, count=len(b.segments))
        per_req = np.array([(r.a, r.b, r.L) for r, _, _ in b.segments], dtype=np.int32)
        b.a = np.repeat(per_req[:, 0], counts)
        b.b = np.repeat(per_req[:, 1], counts)
        b.L = np.repeat(per_req[:, 2], counts)
        b.rot = np.concatenate([r.rot[k:k + t] for r, k, t in b.segments])
        b.R0 = np.concatenate([r.R0[k:k + t] for r, k, t in b.segments])
        return b

    def _complete(self, handle, batch):
        E, st = self.ex.collect(handle)
        now = self.clock()
        off = 0
        for req, k, t in batch.segments:
            if req.state == "active":  # else cancelled meanwhile: results discarded
                req.E[k:k + t] = E[off:off + t]
                req.status[k:k + t] = st[off:off + t]
                req.done_items += t
                if req.done_items == req.n:
                    req.state = "done"
                    req.t_done = now
                    self.active.remove(req)
                    self.used -= req.footprint
                    self.done.append(req)
            off += t

    def step(self):
        """One scheduling iteration; returns True if anything happened."""
        progressed = False
        while self.inflight and self.ex.ready(self.inflight[0][0]):
            h, bt = self.inflight.popleft()
            self._complete(h, bt)
            progressed = True
        self._admit()
        if len(self.inflight) < self.depth:
            batch = self._pack()
            if len(batch):
                self.inflight.append((self.ex.submit(batch), batch))
                progressed = True
        return progressed

    def busy(self):
        return bool(self.pending or self.active or self.inflight)

    def drain(self):
        while self.busy():
            if not self.step() and self.inflight:
                self.ex.wait(self.inflight[0][0])

    # -- a timed stream
    def run_stream(self, requests, idle_sleep=50e-6):
        """Feed requests at their arrival times (seconds from now) and run until all are served."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        for r in reqs:
            r.arrival += t0
        i = 0
        while i < len(reqs) or self.busy():
            now = self.clock()
            while i < len(reqs) and reqs[i].arrival <= now:
                self.submit(reqs[i])
                i += 1
            if not self.step():
                if self.inflight:
                    time.sleep(idle_sleep)  # poll: arrivals keep being admitted meanwhile
                elif i < len(reqs):
                    time.sleep(min(idle_sleep, max(0.0, reqs[i].arrival - self.clock())))
        return self.metrics(t0)

    def metrics(self, t0):
        lat = np.array([r.t_done - r.arrival for r in self.done])
        t_end = max([r.t_done for r in self.done], default=t0)
        n_items = sum(r.n for r in self.done)
        return {
            "requests_done": len(self.done), "requests_rejected": len(self.rejected),
            "energies": int(n_items), "seconds": t_end - t0,
            "energies_per_s": n_items / max(t_end - t0, 1e-12),
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                           "p99": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                           "max": float(lat.max() * 1e3) if len(lat) else None},
        }


# ----------------------------------------------------------------------------- GPU executor

class GpuExecutor:
    """Runs batches through tcm_energy_batch on a CUDA stream; results come back through pinned
    buffers and an event per batch."""

    def __init__(self, systems, lmax_cap=24, precision=None, device=0, ring=4, rotate_cached=False):
        import torch

        from . import tcm
        self.torch, self.tcm = torch, tcm
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream()
        self.precision = tcm.TCM_MIXED if precision is None else precision
        self.ctx = tcm.Context(lmax_cap=lmax_cap, stream=self.stream)
        # rotated sides from the moment cache (Wigner rotation) instead of B's atoms
        self.rotate_cached = bool(rotate_cached)
        self.ctx.tcm_ctx_set_rotate_cached(self.rotate_cached)
        self.coords = []
        self.descr = []
        self.cache = []
        with torch.cuda.stream(self.stream):
            for s in systems:
                t = torch.tensor(np.asarray(s, dtype=np.float32), device="cuda")
                c, a = self.ctx.tcm_prepare(t)
                m = self.ctx.tcm_moments(t, lmax_cap, precision=self.precision, center=c, radius=a)
                self.coords.append(t)
                self.cache.append(m)
                self.descr.append(tcm.make_system(t, center=c, radius=a, moments=m))
        torch.cuda.synchronize()
        self.radius = np.array([d.radius for d in self.descr])
        self.natoms = np.array([len(s) for s in systems])
        self.sys_arr = (tcm.tcm_system * len(self.descr))(*self.descr)
        self.ring = [self._slot(4096) for _ in range(ring)]
        self.slot = 0

    def _slot(self, n):
        t = self.torch
        return {"E": t.empty(n, dtype=t.float64, device="cuda"), "st": t.empty(n, dtype=t.int32, device="cuda"),
                "Eh": t.empty(n, dtype=t.float64).pin_memory(), "sth": t.empty(n, dtype=t.int32).pin_memory(),
                "ev": t.cuda.Event(), "busy": False}

    def submit(self, batch):
        tcm, t = self.tcm, self.torch
        k = len(batch)
        sl = self.ring[self.slot]
        self.slot = (self.slot + 1) % len(self.ring)
        if sl["busy"]:
            sl["ev"].synchronize()
        if sl["E"].numel() < k:
            sl.update(self._slot(max(k, 2 * sl["E"].numel())))
        items = np.zeros(k, dtype=tcm.PAIR_ITEM_DTYPE)
        items["a"] = batch.a
        items["b"] = batch.b
        items["lmax"] = batch.L
        items["has_rot"] = 1
        items["rotB"] = np.asarray(batch.rot).reshape(k, 9)
        items["R0"] = np.asarray(batch.R0).reshape(k, 3)
        pb = tcm.PackedBatch(self.sys_arr, len(self.descr), items, [])
        with t.cuda.stream(self.stream):
            self.ctx.tcm_energy_batch_packed(pb, self.precision, sl["E"], sl["st"])
            sl["Eh"][:k].copy_(sl["E"][:k], non_blocking=True)
            sl["sth"][:k].copy_(sl["st"][:k], non_blocking=True)
            sl["ev"].record(self.stream)
        sl["busy"] = True
        return (sl, k)

    def ready(self, h):
        return h[0]["ev"].query()

    def wait(self, h):
        h[0]["ev"].synchronize()

    def collect(self, h):
        sl, k = h
        sl["ev"].synchronize()
        sl["busy"] = False
        return sl["Eh"][:k].numpy().copy(), sl["sth"][:k].numpy().copy()

    def item_bytes(self, req):
        """Device bytes of one in-flight item: B's moment set, its tile partials, the energy (only
        the descriptor and the energy when B's moments come rotated from the cache)."""
        if self.rotate_cached:
            return 128 + 16 + 256
        nch = max(1, ((req.L + 1) ** 2 + 159) // 160)
        tiles = max(1, -(-int(self.natoms[req.b]) // 2048))
        return 8 * (req.L + 1) ** 2 + 8 * 160 * nch * tiles + 16 + 256


def make_requests(stream, seconds=None):
    """Requests of a synth.ServeStream (rotations and R0 from each request's own seed)."""
    from . import synth
    rad = np.array([synth.centroid_and_radius(s)[1] for s in stream.systems])
    reqs = []
    for i in range(len(stream.arrivals)):
        if seconds is not None and stream.arrivals[i] > seconds:
            break
        a, b = int(stream.pair_a[i]), int(stream.pair_b[i])
        rot, R0 = synth.request_orientations(stream.rot_seed[i], int(stream.n_orient[i]), rad[a] + rad[b])
        reqs.append(Request(i, a, b, int(stream.L[i]), rot, R0, arrival=float(stream.arrivals[i])))
    return reqs


def plain_fp64(ex, reqs):
    """The same requests one at a time through the single-request FP64 calls (tcm_moments per
    side and orientation, tcm_energy), no batching; returns (energies/s, atom-moments/s)."""
    tcm, torch = ex.tcm, ex.torch
    ctx = tcm.Context(lmax_cap=24)
    n_e = 0
    atoms = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        da, db = ex.descr[r.a], ex.descr[r.b]
        ma = ctx.tcm_moments(ex.coords[r.a], r.L, precision=tcm.TCM_FP64, center=da.center, radius=da.radius)
        for k in range(r.n):
            mb = ctx.tcm_moments(ex.coords[r.b], r.L, precision=tcm.TCM_FP64, rot=r.rot[k], center=db.center,
                                 radius=db.radius)
            ctx.tcm_energy(ma, mb, r.R0[k], r.L)
        n_e += r.n
        atoms += ex.natoms[r.a] + r.n * ex.natoms[r.b]
    dt = time.perf_counter() - t0
    ctx.close()
    return n_e / dt, atoms / dt


def main():
    p = argparse.ArgumentParser(description="serve a Poisson stream of TCM scan requests on one GPU")
    p.add_argument("--seconds", type=float, default=10.0)
    p.add_argument("--rate", type=float, default=2000.0)
    p.add_argument("--pool", type=int, default=512)
    p.add_argument("--max-items", type=int, default=8192)
    p.add_argument("--quota", type=int, default=512)
    p.add_argument("--budget-gb", type=float, default=4.0)
    p.add_argument("--plain-fp64", type=int, default=100, help="requests timed through the plain FP64 path")
    p.add_argument("--rotate-cached", action="store_true",
                   help="rotate B's cached moments per orientation instead of recomputing them from its atoms")
    args = p.parse_args()
    from . import synth
    st = synth.serve_stream(n_pool=args.pool, rate=args.rate, seconds=args.seconds)
    ex = GpuExecutor(st.systems, rotate_cached=args.rotate_cached)
    eng = Engine(ex, ex.item_bytes, budget_bytes=int(args.budget_gb * (1 << 30)), max_items=args.max_items,
                 quota=args.quota)
    reqs = make_requests(st)
    atom_moments = sum(r.n * ex.natoms[r.b] for r in reqs)
    m = eng.run_stream(reqs)
    m["atom_moments_per_s"] = None if args.rotate_cached else atom_moments / max(m["seconds"], 1e-12)
    m["workload"] = st.name
    m["offered_requests_per_s"] = args.rate
    m["precision"] = "mixed (float moments, double contraction)"
    m["b_moments"] = "rotated from the cache (Wigner)" if args.rotate_cached else "recomputed from B's atoms"
    if args.plain_fp64 > 0:
        sample = make_requests(st)[:args.plain_fp64]
        e_s, a_s = plain_fp64(ex, sample)
        m["plain_fp64_gpu"] = {"energies_per_s": e_s, "atom_moments_per_s": a_s, "requests": len(sample),
                               "how": "one request at a time: tcm_moments (FP64) per side and orientation + tcm_energy"}
    print(json.dumps(m))


if __name__ == "__main__":
    main()
