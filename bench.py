#!/usr/bin/env python
"""Benchmark of the two-center multipole (TCM) hot path on GB300.

Workload (one "step"): the protein-like PES scan -- systems A and B of 20,000 atoms each
(seeded random-walk chains, bond 1.5 A, confined to r = 30 A, N(0, 0.3) net-zero charges),
256 seeded orientations of B (uniform rotation about its centre, |R0| uniform in
[70, 150] A), Lmax = 20, mixed precision.  One step runs the whole path through the C ABI
(tcm_energy_batch): centre and radius of A and B on the device, the moments of A and of the
256 rotated copies of B (5.14e6 atom-moments), the cross-tile reductions and the 256
two-center contractions.  Inputs are resident in HBM; L2 is flushed (256 MB write, untimed)
before every timed step.

Prints one JSON line (see the design doc for every key).  ``--impl reference`` times the CPU
oracle instead.  Under torchrun each rank runs its own copy of the workload on its GPU
(weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-moments/s and TCM energies/s vs plain FP64 GPU path at stated error; p50/p99"
UNIT = "atom-moments/s"
FP32_LANES_PER_SM = 128
FP64_PER_SM_CLK = 2          # FP64 pipe results per SM per clock (GB300)
DIRECT_FP64_PER_PAIR = 10    # algorithmic FP64 operations per pair of Eq. (Coulomb), besides the rsqrt


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-pes-grid", action="store_true", help="skip the surface-scan measurement")
    return p.parse_args()


# ----------------------------------------------------------------------------- workload

def workload():
    from paper_0704_1672_gb300 import synth
    s = synth.protein_pes_scan()
    k = len(s.R0)
    atoms = len(s.A) + k * len(s.B)
    cfg = {"workload": "protein-like PES scan: 2 x 20000 random-walk atoms (r=30 A, N(0,0.3) net-zero), "
                       "256 orientations of B, |R0| in [70,150] A, Lmax=20",
           "n_atoms_A": len(s.A), "n_atoms_B": len(s.B), "orientations": k, "lmax": s.L,
           "atom_moments_per_step": atoms, "energies_per_step": k, "coords": "float32 (x,y,z,q)",
           "l2": "flushed before every timed step (256 MB write, untimed); inputs 640 KB"}
    return s, atoms, cfg


def captured_traffic(kernel_profile, sources):
    """DRAM bytes per launch from the committed ncu summary, if the kernel sources are unchanged
    since that capture (their hash is recorded in the summary); else None."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", kernel_profile)).read()
    except OSError:
        return None
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_0704_1672_gb300", "csrc", src), "rb").read())
    fields = dict(line.split(":", 1) for line in text.splitlines() if line.startswith(("source_sha256_16:", "traffic_bytes_per_launch:")))
    if fields.get("source_sha256_16", "").split()[0:1] != [h.hexdigest()[:16]]:
        return None
    try:
        return int(fields["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


def moment_instr_per_atom(L):
    """Algorithmic FP32-pipe instructions per atom-moment at order L (3 per real component + 12)."""
    return 3 * (L + 1) ** 2 + 12


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle leg

def oracle_calibrate(s):
    """Seconds per atom of the oracle's Eq. (multipole) at the workload's L (single thread)."""
    import oracle
    cB, _ = oracle.center_radius(s.B)
    t0 = time.perf_counter()
    oracle.moments(s.B[:200], cB, s.L, rot=s.rotB[0])
    return (time.perf_counter() - t0) / 200


def oracle_contraction_seconds(s):
    """One Eq. (Formula) contraction at the workload's L by the oracle (single thread)."""
    import oracle
    cA, _ = oracle.center_radius(s.A)
    cB, _ = oracle.center_radius(s.B)
    QA = oracle.moments(s.A[:50], cA, s.L)
    QB = oracle.moments(s.B[:50], cB, s.L)
    t0 = time.perf_counter()
    oracle.tcm_energy(s.L, QA, QB, s.R0[0])
    return time.perf_counter() - t0


def oracle_step(s, n, threads, pool):
    """Oracle (as it stands) on a bounded sample of the workload: Eq. (multipole) of rotated B
    over the first n atoms, split across host threads.  Returns wall seconds."""
    import oracle
    cB, _ = oracle.center_radius(s.B)
    bounds = np.linspace(0, n, threads + 1).astype(int)
    t0 = time.perf_counter()
    futs = [pool.submit(oracle.moments, s.B[bounds[i]:bounds[i + 1]], cB, s.L, s.rotB[1]) for i in range(threads)]
    for f in futs:
        f.result()
    return time.perf_counter() - t0


def cpu_model():
    """The host CPU's model name (lscpu), for the baseline line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_direct_pairs_per_s(s, threads, pool, n_a=400):
    """Eq. (Coulomb) by the oracle on a sample: the first n_a atoms of A against all of B, split
    across host threads.  Returns pair interactions per second."""
    import oracle
    cA, _ = oracle.center_radius(s.A)
    cB, _ = oracle.center_radius(s.B)
    bounds = np.linspace(0, n_a, threads + 1).astype(int)
    t0 = time.perf_counter()
    futs = [pool.submit(oracle.direct, s.A[bounds[i]:bounds[i + 1]], cA, s.B, cB, s.R0[0], s.rotB[0])
            for i in range(threads)]
    for f in futs:
        f.result()
    return n_a * len(s.B) / (time.perf_counter() - t0)


def oracle_sample_size(per_atom, seconds, threads, n_max):
    return int(min(n_max, max(threads * 8, seconds * threads / per_atom)))


def run_reference(args, rank, world):
    from concurrent.futures import ThreadPoolExecutor
    if rank != 0:
        return
    s, atoms_per_step, cfg = workload()
    threads = os.cpu_count() or 1
    per_atom = oracle_calibrate(s)
    t_con = oracle_contraction_seconds(s)
    budget = min(0.5, 120.0 / max(1, args.steps + args.warmup))
    n = oracle_sample_size(per_atom, budget, threads, len(s.B))
    with ThreadPoolExecutor(max_workers=threads) as pool:
        for _ in range(args.warmup):
            oracle_step(s, n, threads, pool)
        times = [oracle_step(s, n, threads, pool) for _ in range(args.steps)]
    tot_t = float(sum(times))
    value = n * args.steps / tot_t
    sample = (f"per step: oracle Eq. (multipole) at L={s.L} over {n} atoms of rotated B split across {threads} host "
              f"threads; one Eq. (Formula) contraction at L={s.L} takes {t_con:.3f} s single-threaded "
              f"(timed once, not in the steps)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "energies_per_s_single_thread": 1.0 / t_con},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our leg

def run_ours(args, rank, world, dist):
    import torch

    from paper_0704_1672_gb300 import build, tcm
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    s, atoms_per_step, cfg = workload()
    k = len(s.R0)
    L = s.L
    prec = tcm.TCM_MIXED if args.precision == "mixed" else tcm.TCM_FP64
    A = torch.tensor(s.A, dtype=torch.float32, device="cuda")
    B = torch.tensor(s.B, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = tcm.Context(lmax_cap=L, stream=stream)
    # the moment pass's warp-tile size and grid chosen by the library's autotuner on this batch,
    # before any timed step (the batching pillar: tiles chosen by timing, not by a constant)
    from paper_0704_1672_gb300 import autotune
    tuned = autotune.tune(ctx, [(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int),
                          np.full(k, L), s.R0, rotB=s.rotB, precision=prec)
    tiling = {"lmax": L, "atoms_per_lane": tuned.best[L][0], "ctas_per_sm": tuned.best[L][1],
              "moment_phase_ms_by_candidate": {f"{a}x{c}": round(ms, 5) for (a, c), ms in tuned.timings[L].items()}}
    pb = tcm.pack_batch([(A, None, None), (B, None, None)], np.zeros(k, int), np.ones(k, int), np.full(k, L),
                        s.R0, rotB=s.rotB)
    E = torch.empty(k, dtype=torch.float64, device="cuda")
    st = torch.empty(k, dtype=torch.int32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        ctx.tcm_energy_batch_packed(pb, prec, E, st)

    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert bool(torch.all(st == 0)), "non-converged items in the benchmark workload"
    ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(True)

    clocks = ClockSampler(dev)
    if not args.no_clocks:
        clocks.start()
        time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop() if not args.no_clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    phase_ms, launches = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * atoms_per_step * args.steps / (total_ms * 1e-3)
    energies_per_s = world * k * args.steps / (total_ms * 1e-3)

    # roofline of the dominant kernel (moment accumulation, FP32 pipe)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tinstr = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    mom_ms = phase_ms["moments"] / args.steps
    mom_launch_ms = phase_ms["moments"] / max(1, launches["moments"])
    instr = atoms_per_step * moment_instr_per_atom(L) / max(1, launches["moments"] / args.steps)
    achieved = instr / (mom_launch_ms * 1e-3) / 1e12
    traffic = captured_traffic("k_moments_pes_scan_L20.md", ["moments_kernel.cuh", "tcm_internal.h"]) \
        if (L == 20 and prec == tcm.TCM_MIXED) else None
    roofline = {"bound": "alu", "kernel": f"k_moments<float,{L}>", "achieved": achieved, "peak": peak_tinstr,
                "unit": "T FP32-pipe lane-instr/s", "frac": achieved / peak_tinstr, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu, profiles/k_moments_pes_scan_L20.md)",
                "peak_source": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz (max SM clock of measured)",
                "algorithmic_instr_per_atom": moment_instr_per_atom(L)}
    phases = {p: phase_ms[p] / args.steps for p in phase_ms}

    # the same steps with the library's default launch mode, a replayed CUDA graph of the launch
    # sequence (phase timing off: no events between the kernels)
    g_steps = min(args.steps, 500)
    for _ in range(3):
        flush.zero_()
        step()
    evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(g_steps)]
    torch.cuda.synchronize()
    for i in range(g_steps):
        flush.zero_()
        evg[i][0].record(stream)
        step()
        evg[i][1].record(stream)
    torch.cuda.synchronize()
    g_ms = float(sum(a.elapsed_time(b) for a, b in evg)) / g_steps
    g_cap, g_launch = ctx.tcm_ctx_graph_stats()
    graph_replay = {"ms_per_step": g_ms, "value": world * atoms_per_step / (g_ms * 1e-3), "unit": UNIT,
                    "steps": g_steps, "graph_captures": g_cap, "graph_launches": g_launch}

    # the same orientations with B's moments rotated from a cache (Wigner rotation in the
    # contraction kernel) instead of recomputed from its atoms: moments of A and B once, outside
    # the timed steps
    rc_ctx = tcm.Context(lmax_cap=L, stream=stream)
    mA = rc_ctx.tcm_moments(A, L, precision=prec)
    mB = rc_ctx.tcm_moments(B, L, precision=prec)
    rc_pb = tcm.pack_batch([tcm.make_system(A, mA.center, mA.radius, moments=mA),
                            tcm.make_system(B, mB.center, mB.radius, moments=mB)],
                           np.zeros(k, int), np.ones(k, int), np.full(k, L), s.R0, rotB=s.rotB)
    rc_ctx.tcm_ctx_set_rotate_cached(True)
    for _ in range(3):
        flush.zero_()
        rc_ctx.tcm_energy_batch_packed(rc_pb, prec, E, st)
    evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(g_steps)]
    torch.cuda.synchronize()
    for i in range(g_steps):
        flush.zero_()
        evr[i][0].record(stream)
        rc_ctx.tcm_energy_batch_packed(rc_pb, prec, E, st)
        evr[i][1].record(stream)
    torch.cuda.synchronize()
    rc_ms = float(sum(a.elapsed_time(b) for a, b in evr)) / g_steps
    rotate_cached = {"ms_per_step": rc_ms, "energies_per_s": world * k / (rc_ms * 1e-3), "steps": g_steps,
                     "how": "B's cached moments rotated per orientation by Wigner matrices in the contraction "
                            "kernel (O(L^3)); no atom pass per step"}
    rc_ctx.close()

    # the surface scan of Section IV: every grid point at several Lmax from cached moments,
    # and the exact energy of every grid point by the batched direct-sum kernel
    pes_grid = None
    if not args.no_pes_grid and rank == 0:
        pes_grid = run_pes_grid(torch, tcm, prec, n_sm, sm_max_mhz(), stream)

    # end to end through the C ABI with host buffers: H2D of the coordinates, D2H of the energies
    e2e = None
    if args.e2e_steps > 0:
        A_h = torch.tensor(s.A, dtype=torch.float32).pin_memory()
        B_h = torch.tensor(s.B, dtype=torch.float32).pin_memory()
        E_h = torch.empty(k, dtype=torch.float64).pin_memory()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(args.e2e_steps + 3):
            if i == 3:
                torch.cuda.synchronize()
                e0.record(stream)
                t_wall = time.perf_counter()
            A.copy_(A_h, non_blocking=True)
            B.copy_(B_h, non_blocking=True)
            step()
            E_h.copy_(E, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
        e2e = {"value": world * atoms_per_step / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(A_h.numel() * 4 + B_h.numel() * 4),
               "d2h_bytes_per_step": int(E_h.numel() * 8), "ms_per_step": e2e_ms,
               "wall_ms_per_step": 1e3 * t_wall / args.e2e_steps}

    # reference points: the plain single-request FP64 GPU path, and the CPU oracle
    fp64_plain = None
    fp64_batched = None
    if args.fp64_steps > 0 and rank == 0:
        fp64_plain = plain_fp64(ctx, tcm, torch, A, B, s, args.fp64_steps)
        if prec == tcm.TCM_MIXED:
            fp64_batched = batched_fp64(ctx, tcm, torch, pb, E, st, stream, flush, atoms_per_step, k,
                                        n_sm, sm_max, L)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        from concurrent.futures import ThreadPoolExecutor
        threads = os.cpu_count() or 1
        n = len(s.B)
        with ThreadPoolExecutor(max_workers=threads) as pool:
            tm = min(oracle_step(s, n, threads, pool) for _ in range(2))
            t1 = oracle_step(s, n // 8, 1, pool)  # one thread on an eighth of the atoms
            dpairs = oracle_direct_pairs_per_s(s, threads, pool)
        tc = oracle_contraction_seconds(s)
        cpu = {"value": n / tm, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"oracle Eq. (multipole) at L={L} over all {n} atoms of one rotated copy of B, split across "
                         f"{threads} host threads (best of 2); one Eq. (Formula) contraction took {tc:.3f} s "
                         f"single-threaded",
               "single_thread_value": (n // 8) / t1,
               "energies_per_s_single_thread": 1.0 / tc,
               "direct_pairs_per_s": dpairs}

    if rank == 0:
        p50 = float(np.percentile(step_ms, 50))
        p99 = float(np.percentile(step_ms, 99))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if prec == tcm.TCM_MIXED else "f64", "data": "synthetic",
                "config": cfg, "energies_per_s": energies_per_s,
                "step_latency_ms": {"p50": p50, "p99": p99},
                "phase_ms_per_step": phases, "gpu_launches": int(sum(launches.values())),
                "gpu_launches_per_step": {p: launches[p] / args.steps for p in launches},
                "roofline": roofline, "tiling": tiling, "clocks": ck, "e2e": e2e, "graph_replay": graph_replay,
                "rotate_cached": rotate_cached, "pes_grid": pes_grid,
                "fp64_plain_gpu": fp64_plain, "fp64_batched_gpu": fp64_batched,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()


def sm_max_mhz():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def run_pes_grid(torch, tcm, prec, n_sm, sm_mhz, stream):
    """Surface scan (Section IV shapes): 43 x 360 grid in the xy-plane, Lmax in {1,2,3,4,6,8,10},
    TCM energies from cached moments and exact energies at every point."""
    from paper_0704_1672_gb300 import pes, synth
    g = synth.pes_grid_pair()
    A = torch.tensor(g.A, device="cuda")
    B = torch.tensor(g.B, device="cuda")
    R0 = g.R0()
    ctx = tcm.Context(lmax_cap=max(g.lmax), stream=stream)
    try:
        pes.scan(ctx, A, B, R0[:64], g.lmax, precision=prec)  # warm-up (kernel attributes)
        for _ in range(4):  # descriptor staging buffers and scratch at the full grid's size
            pes.scan(ctx, A, B, R0, g.lmax, precision=prec, direct=False)
        res = pes.scan(ctx, A, B, R0, g.lmax, precision=prec)
    finally:
        ctx.close()
    n = len(R0)
    t = res.timings_ms
    pairs = n * len(g.A) * len(g.B)
    achieved = pairs * DIRECT_FP64_PER_PAIR / (t["direct"] * 1e-3) / 1e9
    peak = n_sm * FP64_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    return {"workload": g.name, "points": n, "lmax": list(g.lmax),
            "tcm_energies": n * len(g.lmax), "tcm_ms": t["tcm_energies"], "moments_ms": t["moments"],
            "item_packing_host_ms": t["item_packing_host"],
            "tcm_energies_per_s": n * len(g.lmax) / (t["tcm_energies"] * 1e-3),
            "direct_ms": t["direct"], "direct_pairs_per_s": pairs / (t["direct"] * 1e-3),
            "direct_roofline": {"bound": "fp64", "kernel": "k_direct", "achieved": achieved, "peak": peak,
                                "unit": "G FP64 op/s", "frac": achieved / peak,
                                "algorithmic_fp64_per_pair": DIRECT_FP64_PER_PAIR,
                                "peak_source": f"{n_sm} SMs x {FP64_PER_SM_CLK} FP64/clk x {sm_mhz:.0f} MHz"},
            "eq_error_percent_median": {str(L): float(np.median(res.eta(L))) for L in g.lmax},
            "eq_error_percent_max": {str(L): float(np.max(res.eta(L))) for L in g.lmax}}


def batched_fp64(ctx, tcm, torch, pb, E, st, stream, flush, atoms_per_step, k, n_sm, sm_mhz, L, steps=5):
    """The same batched step in double precision throughout (double moment kernels): the
    accuracy the plain FP64 path has, at batched throughput.  Moment phase against the FP64
    pipe (3 (L+1)^2 + 12 FP64 instructions per atom-moment)."""
    ctx.tcm_ctx_set_profiling(True)
    ctx.tcm_ctx_read_profile()
    for _ in range(2):
        flush.zero_()
        ctx.tcm_energy_batch_packed(pb, tcm.TCM_FP64, E, st)
    torch.cuda.synchronize()
    ctx.tcm_ctx_read_profile()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        ctx.tcm_energy_batch_packed(pb, tcm.TCM_FP64, E, st)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms, launches = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    step_ms = tot / steps
    mom_ms = ms["moments"] / max(1, launches["moments"])
    achieved = atoms_per_step * moment_instr_per_atom(L) / (mom_ms * 1e-3) / 1e9
    peak = n_sm * FP64_PER_SM_CLK * sm_mhz * 1e6 / 1e9
    return {"value": atoms_per_step / (step_ms * 1e-3), "unit": UNIT, "energies_per_s": k / (step_ms * 1e-3),
            "ms_per_step": step_ms, "steps": steps, "moments_ms": mom_ms,
            "moments_roofline": {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "G FP64 instr/s",
                                 "frac": achieved / peak},
            "how": "the benchmark batch through tcm_energy_batch at TCM_FP64 (double moment kernels)"}


def plain_fp64(ctx, tcm, torch, A, B, s, steps):
    """The plain FP64 GPU path: one request at a time through tcm_moments + tcm_energy, no batching."""
    k = len(s.R0)
    L = s.L
    qA = torch.empty((L + 1) ** 2, dtype=torch.float64, device="cuda")
    qB = torch.empty((L + 1) ** 2, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    for _ in range(steps):
        ma = ctx.tcm_moments(A, L, precision=tcm.TCM_FP64, out=qA)
        for i in range(k):
            mb = ctx.tcm_moments(B, L, precision=tcm.TCM_FP64, rot=s.rotB[i], out=qB)
            ctx.tcm_energy(ma, mb, s.R0[i], L)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    atoms = len(s.A) + k * len(s.B)
    return {"value": atoms / dt, "unit": UNIT, "energies_per_s": k / dt, "ms_per_step": 1e3 * dt, "steps": steps,
            "how": "per orientation: tcm_moments(B, FP64, rotated) + tcm_energy (synchronous); A once per step"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
