#!/usr/bin/env python
"""Benchmark of the two-center multipole (TCM) hot path on GB300.

Headline workload (one "step"): the large assembly -- A = 1,000,000 charges +-1 (2 % net
excess) uniform in a shell 80-100 A, B = a 50,000-atom random-walk ligand (bond 1.5 A, radius
1.9 N^(1/3) A, N(0, 0.3) net-zero charges), 10,000 seeded orientations of B (uniform rotation
about its centre, |R0| uniform in [max(150, 1.05 (a_A + a_B)), 300] A), Lmax = 24, B's moments
recomputed from its atoms for every orientation, mixed precision.  One step is one batched call
of the C ABI (tcm_energy_batch): centre, radius and low-degree sums of A and B on the device,
the moments of A and of the 10,000 rotated copies of B (5.01e8 atom-moments at 625
components), the cross-tile reductions and the 10,000 two-center contractions.  Inputs are
resident in HBM; L2 is flushed (256 MB write, untimed) before every timed step.

The same JSON line carries the other workloads: the protein-like PES scan (2 x 20,000 atoms,
256 orientations, Lmax = 20), one call of 4,096 uneven pairs (Lmax in {8, 12, 16, 24}), the
serving stream (Poisson arrivals at 2,000 requests/s for 60 s over 512 resident systems), the
surface scan of Section IV, the plain single-request FP64 GPU path and the CPU oracle.
``--impl reference`` times the CPU oracle instead.  Under torchrun each rank runs its own copy
of the workload on its GPU (weak scaling, no collective on the data path).
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
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--no-extras", action="store_true", help="headline workload only")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-pes-grid", action="store_true", help="skip the surface-scan measurement")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--only", choices=["protein_pes_scan", "uneven_pairs"], default=None,
                   help="run one of the other workloads alone and print its record (for profiling captures)")
    p.add_argument("--tiling", default=None, metavar="APL,CTAS,KMAX",
                   help="apply this moment-pass tiling instead of running the autotuner (for profiling captures "
                        "of the tuned launch configuration)")
    p.add_argument("--orientations", type=int, default=10000,
                   help="orientations of B in the headline workload (10,000; fewer only for profiling captures)")
    return p.parse_args()


# ----------------------------------------------------------------------------- work counts

def moment_instr_per_atom(L):
    """Algorithmic FP32-pipe instructions per atom-moment at order L (3 per real component + 12)."""
    return 3 * (L + 1) ** 2 + 12


def contract_fp64_ops(L):
    """Algorithmic FP64 operations of one energy in k_contract when B's moments arrive in the
    frame of R0 and A's are rotated in the kernel: the input and beta phases and the scalings of
    the (l, m >= 0) entries (12 per entry), the two products through d^l(pi/2)
    (2 sum_l (l+1)^2), the z-axis contraction (sum over (l1, l2) of 2 min(l1, l2), plus 3 per
    pair) and the power tables (about 250)."""
    T = (L + 1) * (L + 2) // 2
    S2 = (L + 1) * (L + 2) * (2 * L + 3) // 6
    Z = sum(2 * min(a, b) for a in range(L + 1) for b in range(L + 1))
    return 12 * T + 2 * S2 + Z + 3 * (L + 1) ** 2 + 250


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def sm_max_mhz():
    return float(measured_peaks().get("sm_max_mhz", 2070.0))


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
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("source_sha256_16:", "traffic_bytes_per_launch:")))
    if fields.get("source_sha256_16", "").split()[0:1] != [h.hexdigest()[:16]]:
        return None
    try:
        return int(fields["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


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
        return self

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


def no_clocks():
    return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"], "samples": 0}


# ----------------------------------------------------------------------------- oracle legs

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


def oracle_moments_split(pool, threads, X, c, L, rot=None):
    """The oracle's Eq. (multipole) over X split across host threads (ctypes releases the GIL)."""
    import oracle
    bounds = np.linspace(0, len(X), threads + 1).astype(int)
    futs = [pool.submit(oracle.moments, X[bounds[i]:bounds[i + 1]], c, L, rot) for i in range(threads)
            if bounds[i + 1] > bounds[i]]
    out = None
    for f in futs:
        q = f.result()
        out = q if out is None else out + q
    return out


def oracle_pair_sample(pool, threads, A, B, rots, R0s, L, a_frac=1.0):
    """The oracle as it stands on a sample of a pair-scan workload: Eq. (multipole) of A (on the
    first a_frac of its atoms, scaled to all of them), of B under each sampled rotation (all
    atoms, split across threads) and one Eq. (Formula) contraction per sampled orientation
    (the contractions of the sample run in parallel, one per thread).  Returns (seconds per
    orientation excluding A, seconds for all of A's moments, seconds per contraction)."""
    import oracle
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    na = max(threads, int(len(A) * a_frac))
    t0 = time.perf_counter()
    QA = oracle_moments_split(pool, threads, A[:na], cA, L)
    tA = (time.perf_counter() - t0) * len(A) / na
    t0 = time.perf_counter()
    QBs = [oracle_moments_split(pool, threads, B, cB, L, rot) for rot in rots]
    tB = (time.perf_counter() - t0) / len(rots)
    t0 = time.perf_counter()
    futs = [pool.submit(oracle.tcm_energy, L, QA, QB, R0) for QB, R0 in zip(QBs, R0s)]
    for f in futs:
        f.result()
    tC = (time.perf_counter() - t0) * min(threads, len(rots)) / len(rots)  # per contraction, one thread
    return tB, tA, tC


def cpu_baselines(s4, threads, pool, budget_s=8.0):
    """The CPU oracle on bounded samples of every workload, all host threads and one thread.
    Every figure is a sample, extrapolated to the workload's unit and labelled."""
    import oracle
    from paper_0704_1672_gb300 import synth
    out = {"cores": threads, "cpu_model": cpu_model(), "kind": "oracle"}
    # single pair (Section III shape): in full
    s1 = synth.single_pair_sphere()
    cA, _ = oracle.center_radius(s1.A)
    cB, _ = oracle.center_radius(s1.B)
    t0 = time.perf_counter()
    QA, QB = oracle.moments(s1.A, cA, s1.L), oracle.moments(s1.B, cB, s1.L)
    oracle.tcm_energy(s1.L, QA, QB, s1.R0[0])
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.direct(s1.A, cA, s1.B, cB, s1.R0[0])
    td = time.perf_counter() - t0
    out["single_pair_L10"] = {"energies_per_s": 1.0 / t1, "seconds_per_energy": t1, "direct_seconds": td,
                              "threads": 1, "sample": "the whole workload (2 x 200 charges, one energy), one thread"}
    # large assembly (headline): 2 orientations of B with their contractions, A on 1/64 of its atoms
    k = 2
    tB, tA, tC = oracle_pair_sample(pool, threads, s4.A, s4.B, s4.rotB[:k], s4.R0[:k], s4.L, a_frac=1 / 64)
    n_or = len(s4.R0)
    t_step = tA + n_or * (tB + tC / threads)
    atoms = len(s4.A) + n_or * len(s4.B)
    out["large_assembly_L24"] = {
        "value": atoms / t_step, "unit": UNIT, "energies_per_s": n_or / t_step, "threads": threads,
        "seconds_per_orientation": tB + tC / threads, "seconds_A_moments": tA, "seconds_per_contraction_1thread": tC,
        "sample": f"{k} orientations of B (all 50,000 atoms, split across {threads} threads) with their Eq. (Formula) "
                  f"contractions, A's moments on 1/64 of its atoms; extrapolated to the 10,000-orientation step"}
    # one thread on a slice of B (per-atom rate)
    cB, _ = oracle.center_radius(s4.B)
    n1 = 400
    t0 = time.perf_counter()
    oracle.moments(s4.B[:n1], cB, s4.L, s4.rotB[0])
    t1a = (time.perf_counter() - t0) / n1
    out["large_assembly_L24"]["single_thread_value"] = 1.0 / (t1a + tC / len(s4.B))
    # protein-like scan: 2 orientations with contractions
    s2 = synth.protein_pes_scan()
    tB2, tA2, tC2 = oracle_pair_sample(pool, threads, s2.A, s2.B, s2.rotB[:2], s2.R0[:2], s2.L)
    t2 = tA2 + len(s2.R0) * (tB2 + tC2 / threads)
    out["protein_pes_scan_L20"] = {
        "value": (len(s2.A) + len(s2.R0) * len(s2.B)) / t2, "unit": UNIT, "energies_per_s": len(s2.R0) / t2,
        "threads": threads, "seconds_per_contraction_1thread": tC2,
        "sample": f"2 of 256 orientations (B's moments split across {threads} threads, contractions), A in full; "
                  f"extrapolated to the 256-orientation step"}
    # uneven pairs: the 16 smallest-L items of a seeded sample
    b3 = synth.uneven_batch(n_pairs=64, seed=3)
    t0 = time.perf_counter()
    am = 0
    futs = []
    for i in range(16):
        A3, B3 = b3.systems[b3.pair_a[i]], b3.systems[b3.pair_b[i]]
        futs.append(pool.submit(_oracle_item, A3, B3, int(b3.L[i]), b3.rotB[i], b3.R0[i]))
        am += len(A3) + len(B3)
    for f in futs:
        f.result()
    t3 = time.perf_counter() - t0
    out["uneven_pairs"] = {"value": am / t3, "unit": UNIT, "energies_per_s": 16 / t3, "threads": threads,
                           "sample": "16 pairs of a 64-pair draw of the uneven workload (same distributions), one "
                                     "pair per thread: moments of both sides and the contraction"}
    return out


def _oracle_item(A, B, L, rot, R0):
    import oracle
    cA, _ = oracle.center_radius(A)
    cB, _ = oracle.center_radius(B)
    return oracle.tcm_energy(L, oracle.moments(A, cA, L), oracle.moments(B, cB, L, rot), R0)


def run_reference(args, rank, world):
    """The CPU oracle as it stands on the headline workload: each step is a bounded sample (one
    orientation of B: its moments over all of B's atoms split across the host threads, and its
    Eq. (Formula) contraction), reported per atom-moment of the step."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_0704_1672_gb300 import synth
    if rank != 0:
        return
    s = synth.large_assembly()
    cfg = config4_cfg(s)
    threads = os.cpu_count() or 1
    cA, _ = oracle.center_radius(s.A)
    cB, _ = oracle.center_radius(s.B)
    with ThreadPoolExecutor(max_workers=threads) as pool:
        QA = oracle_moments_split(pool, threads, s.A[:20000], cA, s.L)  # a fixed stand-in for A (not timed)

        def one(k):
            t0 = time.perf_counter()
            QB = oracle_moments_split(pool, threads, s.B, cB, s.L, s.rotB[k])
            oracle.tcm_energy(s.L, QA, QB, s.R0[k])
            return time.perf_counter() - t0

        for k in range(args.warmup):
            one(k)
        times = [one(args.warmup + k) for k in range(args.steps)]
    tot = float(sum(times))
    value = len(s.B) * args.steps / tot
    sample = (f"per step: one orientation of B -- the oracle's Eq. (multipole) at L={s.L} over all {len(s.B)} atoms "
              f"split across {threads} host threads, and its Eq. (Formula) contraction (one thread)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- timing helpers

class Timer:
    """Times steps with CUDA events on one stream, with an L2 flush (untimed) before each."""

    def __init__(self, torch, stream):
        self.torch = torch
        self.stream = stream
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def run(self, fn, steps, warmup, dist=None):
        torch = self.torch
        for _ in range(warmup):
            self.flush.zero_()
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            self.flush.zero_()
            ev[i][0].record(self.stream)
            fn()
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return [a.elapsed_time(b) for a, b in ev]


def config4_cfg(s):
    atoms = len(s.A) + len(s.R0) * len(s.B)
    return {"workload": "large assembly: A = 1,000,000 charges +-1 (2% excess) in an 80-100 A shell, B = 50,000-atom "
                        f"random-walk ligand, {len(s.R0):,} orientations of B, |R0| in [max(150, 1.05(a_A+a_B)), 300] A, "
                        "Lmax=24, B's moments recomputed per orientation",
            "n_atoms_A": len(s.A), "n_atoms_B": len(s.B), "orientations": len(s.R0), "lmax": s.L,
            "atom_moments_per_step": atoms, "energies_per_step": len(s.R0), "coords": "float32 (x,y,z,q)",
            "l2": "flushed before every timed step (256 MB write, untimed); inputs 16.8 MB"}


# ----------------------------------------------------------------------------- our leg

def run_ours(args, rank, world, dist):
    import torch

    from paper_0704_1672_gb300 import autotune, build, synth, tcm
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    smx = sm_max_mhz()
    peak_fp32 = n_sm * FP32_LANES_PER_SM * smx * 1e6 / 1e12      # T lane-instr/s
    peak_fp64 = n_sm * FP64_PER_SM_CLK * smx * 1e6 / 1e9         # G FP64 op/s
    prec = tcm.TCM_MIXED if args.precision == "mixed" else tcm.TCM_FP64
    stream = torch.cuda.current_stream()
    timer = Timer(torch, stream)

    # ---- headline: large assembly
    s = synth.large_assembly(n_orient=args.orientations)
    k = len(s.R0)
    L = s.L
    cfg = config4_cfg(s)
    atoms_per_step = cfg["atom_moments_per_step"]
    A = torch.tensor(s.A, dtype=torch.float32, device="cuda")
    B = torch.tensor(s.B, dtype=torch.float32, device="cuda")
    ctx = tcm.Context(lmax_cap=24, stream=stream)
    systems = [(A, None, None), (B, None, None)]
    ia, ib, il = np.zeros(k, int), np.ones(k, int), np.full(k, L)
    tiling = None
    if args.tiling:
        tiling = fixed_tiling(ctx, tcm, prec, L, args.tiling)
    elif not args.no_autotune:
        # the moment pass's warp tiles, grid and L-chunking chosen by the library's autotuner on a
        # sample of this batch's own items, before any timed step
        tuned = autotune.tune(ctx, systems, ia, ib, il, s.R0, rotB=s.rotB, precision=prec, reps=2,
                              max_items_per_l=1024, atoms_per_lane=(32, 64, 96, 128, 256, 512))
        tiling = {"lmax": L, "atoms_per_lane": tuned.best[L][0], "ctas_per_sm": tuned.best[L][1],
                  "kmax": tuned.best[L][2], "chunks": ctx.tcm_ctx_get_chunking_l(L)[1],
                  "tuned_on": "1,024 of the 10,000 orientations",
                  "moment_phase_ms_by_candidate": {"x".join(str(x) for x in c): round(ms, 5)
                                                   for c, ms in tuned.timings[L].items()},
                  "candidate_key": "atoms_per_lane x ctas_per_sm x kmax"}
    pb = tcm.pack_batch(systems, ia, ib, il, s.R0, rotB=s.rotB)
    E = torch.empty(k, dtype=torch.float64, device="cuda")
    st = torch.empty(k, dtype=torch.int32, device="cuda")

    def step():
        ctx.tcm_energy_batch_packed(pb, prec, E, st)

    step()
    torch.cuda.synchronize()
    assert bool(torch.all(st == 0)), "non-converged items in the benchmark workload"
    ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(True)
    clocks = ClockSampler(dev).start() if not args.no_clocks else None
    if clocks:
        time.sleep(0.3)
    step_ms = timer.run(step, args.steps, max(3, args.warmup), dist)
    ck = clocks.stop() if clocks else no_clocks()
    phase_ms, launches = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    # the warm-up steps were profiled too: scale the phase totals to the timed steps
    n_prof = args.steps + max(3, args.warmup)
    total_ms = float(sum(step_ms))
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * atoms_per_step * args.steps / (total_ms * 1e-3)
    energies_per_s = world * k * args.steps / (total_ms * 1e-3)
    phases = {p: phase_ms[p] / n_prof for p in phase_ms}
    launches_per_step = {p: launches[p] / n_prof for p in launches}
    mom_launch_ms = phase_ms["moments"] / max(1, launches["moments"])
    instr = atoms_per_step * moment_instr_per_atom(L) / max(1, launches_per_step["moments"])
    achieved = instr / (mom_launch_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": f"k_moments<float,{L}>", "achieved": achieved, "peak": peak_fp32,
                "unit": "T FP32-pipe lane-instr/s", "frac": achieved / peak_fp32,
                "traffic": captured_traffic(f"k_moments_large_assembly_L{L}.md", ["moments_kernel.cuh", "tcm_internal.h"]),
                "traffic_unit": f"DRAM bytes per launch (ncu, profiles/k_moments_large_assembly_L{L}.md)",
                "peak_source": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {smx:.0f} MHz (max SM clock of measured)",
                "algorithmic_instr_per_atom": moment_instr_per_atom(L), "launch_ms": mom_launch_ms}
    con_launch_ms = phase_ms["contract"] / max(1, launches["contract"])
    con_ops = k * contract_fp64_ops(L)
    contract_roofline = {"bound": "fp64", "kernel": "k_contract<false>", "achieved": con_ops / (con_launch_ms * 1e-3) / 1e9,
                         "peak": peak_fp64, "unit": "G FP64 op/s",
                         "frac": con_ops / (con_launch_ms * 1e-3) / 1e9 / peak_fp64,
                         "algorithmic_fp64_per_energy": contract_fp64_ops(L), "launch_ms": con_launch_ms,
                         "peak_source": f"{n_sm} SMs x {FP64_PER_SM_CLK} FP64/clk x {smx:.0f} MHz"}

    # the same steps with the library's default launch mode (phase events off: a replayed CUDA graph)
    g_ms = timer.run(step, min(args.steps, 10), 3)
    g_cap, g_launch = ctx.tcm_ctx_graph_stats()
    graph_replay = {"ms_per_step": float(np.mean(g_ms)), "value": world * atoms_per_step / (np.mean(g_ms) * 1e-3),
                    "unit": UNIT, "steps": len(g_ms), "graph_captures": g_cap, "graph_launches": g_launch}

    # end to end through the C ABI with host buffers: H2D of both systems, D2H of the energies
    e2e = None
    if args.e2e_steps > 0:
        A_h = torch.tensor(s.A, dtype=torch.float32).pin_memory()
        B_h = torch.tensor(s.B, dtype=torch.float32).pin_memory()
        E_h = torch.empty(k, dtype=torch.float64).pin_memory()

        def e2e_step():
            A.copy_(A_h, non_blocking=True)
            B.copy_(B_h, non_blocking=True)
            step()
            E_h.copy_(E, non_blocking=True)

        t_wall = time.perf_counter()
        e_ms = timer.run(e2e_step, args.e2e_steps, 2)
        t_wall = time.perf_counter() - t_wall
        e2e_ms = float(np.mean(e_ms))
        e2e = {"value": world * atoms_per_step / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(A_h.numel() * 4 + B_h.numel() * 4),
               "d2h_bytes_per_step": int(E_h.numel() * 8), "ms_per_step": e2e_ms,
               "energies_per_s": world * k / (e2e_ms * 1e-3)}

    extras = {}
    if not args.no_extras and rank == 0:
        extras["protein_pes_scan"] = bench_config2(torch, tcm, synth, autotune, timer, stream, prec, peak_fp32, peak_fp64,
                                                   n_sm, smx)
        extras["uneven_pairs"] = bench_config3(torch, tcm, synth, stream, prec)
        fp64_plain = plain_fp64_config4(ctx, tcm, torch, A, B, s, n_orient=8)
        extras["fp64_plain_gpu"] = fp64_plain
        extras["single_pair"] = bench_config1(torch, tcm, synth)
        if not args.no_serve:
            extras["serving"] = bench_serving(torch, tcm, synth, args.serve_seconds, dev, args.no_clocks)
        if not args.no_pes_grid:
            extras["pes_grid"] = run_pes_grid(torch, tcm, prec, n_sm, smx, stream)
    ctx.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        from concurrent.futures import ThreadPoolExecutor
        threads = os.cpu_count() or 1
        with ThreadPoolExecutor(max_workers=threads) as pool:
            bl = cpu_baselines(s, threads, pool)
        head = bl["large_assembly_L24"]
        cpu = {"value": head["value"], "unit": UNIT, "cores": threads, "kind": "oracle", "sample": head["sample"],
               "cpu_model": bl["cpu_model"], "single_thread_value": head["single_thread_value"],
               "energies_per_s": head["energies_per_s"], "per_workload": bl}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64" if prec == tcm.TCM_MIXED else "f64", "data": "synthetic",
                "config": cfg, "energies_per_s": energies_per_s,
                "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
                "phase_ms_per_step": phases, "gpu_launches": int(round(sum(launches_per_step.values()) * args.steps)),
                "gpu_launches_per_step": launches_per_step,
                "roofline": roofline, "contract_roofline": contract_roofline, "tiling": tiling, "clocks": ck,
                "e2e": e2e, "graph_replay": graph_replay, "cpu_baseline": cpu}
        line.update(extras)
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- other workloads

def fixed_tiling(ctx, tcm, prec, L, spec):
    """Apply an 'APL,CTAS,KMAX' tiling to degree L; returns the record the JSON line carries."""
    apl, cps, km = (int(x) for x in spec.split(","))
    ctx.tcm_ctx_set_tiling_l(prec, L, apl, cps)
    if prec != tcm.TCM_FP64:
        ctx.tcm_ctx_set_chunking_l(L, km)
    return {"lmax": L, "atoms_per_lane": apl, "ctas_per_sm": cps, "kmax": km, "how": "given (--tiling), not tuned"}


def bench_config1(torch, tcm, synth, reps=200):
    """The single pair (2 x 200 charges, Lmax = 10), one energy per call, each call synchronised:
    the plain FP64 path (tcm_moments of both systems, then tcm_energy) and one-item
    tcm_energy_batch calls in FP64 and mixed precision.  Latencies are host wall times per call
    (the work is microseconds; launch and synchronisation dominate)."""
    s = synth.single_pair_sphere()
    A = torch.tensor(s.A, dtype=torch.float64, device="cuda")
    B = torch.tensor(s.B, dtype=torch.float64, device="cuda")
    Af, Bf = A.float(), B.float()
    ctx = tcm.Context(lmax_cap=s.L)
    R0 = np.asarray(s.R0, dtype=np.float64).reshape(1, 3)

    def plain():
        mA = ctx.tcm_moments(A, s.L, precision=tcm.TCM_FP64)
        mB = ctx.tcm_moments(B, s.L, precision=tcm.TCM_FP64)
        return ctx.tcm_energy(mA, mB, R0[0], s.L)

    def batched(prec, X, Y):
        def run():
            E, _ = ctx.tcm_energy_batch([(X, None, None), (Y, None, None)], [0], [1], [s.L], R0, precision=prec)
            return float(E[0])  # device -> host read: the call is synchronised
        return run

    out = {}
    for name, fn in (("fp64_plain", plain), ("fp64_batched", batched(tcm.TCM_FP64, A, B)),
                     ("mixed_batched", batched(tcm.TCM_MIXED, Af, Bf))):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        lat = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            lat.append((time.perf_counter() - t0) * 1e3)
        lat.sort()
        out[name] = {"latency_ms_p50": lat[len(lat) // 2], "latency_ms_p99": lat[int(0.99 * (len(lat) - 1))],
                     "energies_per_s": 1e3 / (sum(lat) / len(lat))}
    ctx.close()
    out["workload"] = "single pair: 2 x 200 charges in r = 10 A spheres, R0 = 40 A, Lmax = 10, one energy per call"
    return out


def bench_config2(torch, tcm, synth, autotune, timer, stream, prec, peak_fp32, peak_fp64, n_sm, smx, steps=200,
                  tune=True, tiling=None):
    """Protein-like PES scan: 2 x 20,000 atoms, 256 orientations of B, Lmax = 20."""
    s = synth.protein_pes_scan()
    k = len(s.R0)
    L = s.L
    atoms = len(s.A) + k * len(s.B)
    A = torch.tensor(s.A, dtype=torch.float32, device="cuda")
    B = torch.tensor(s.B, dtype=torch.float32, device="cuda")
    ctx = tcm.Context(lmax_cap=L, stream=stream)
    systems = [(A, None, None), (B, None, None)]
    ia, ib, il = np.zeros(k, int), np.ones(k, int), np.full(k, L)
    tuned = autotune.tune(ctx, systems, ia, ib, il, s.R0, rotB=s.rotB, precision=prec, reps=3) \
        if (tune and tiling is None) else None
    fixed = fixed_tiling(ctx, tcm, prec, L, tiling) if tiling else None
    pb = tcm.pack_batch(systems, ia, ib, il, s.R0, rotB=s.rotB)
    E = torch.empty(k, dtype=torch.float64, device="cuda")
    st = torch.empty(k, dtype=torch.int32, device="cuda")

    def step():
        ctx.tcm_energy_batch_packed(pb, prec, E, st)

    ctx.tcm_ctx_set_profiling(True)
    ctx.tcm_ctx_read_profile()
    ms = timer.run(step, steps, 5)
    ph, la = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    n = steps + 5
    mom_launch_ms = ph["moments"] / max(1, la["moments"])
    instr = atoms * moment_instr_per_atom(L) / max(1.0, la["moments"] / n)
    ach = instr / (mom_launch_ms * 1e-3) / 1e12
    con_launch_ms = ph["contract"] / max(1, la["contract"])
    con = k * contract_fp64_ops(L) / (con_launch_ms * 1e-3) / 1e9
    g_ms = timer.run(step, steps, 3)
    out = {"workload": "protein-like PES scan: 2 x 20000 random-walk atoms (r=30 A, N(0,0.3) net-zero), 256 "
                       "orientations of B, |R0| in [70,150] A, Lmax=20",
           "atom_moments_per_step": atoms, "energies_per_step": k, "steps": steps,
           "ms_per_step": float(np.mean(ms)), "value": atoms / (np.mean(ms) * 1e-3), "unit": UNIT,
           "energies_per_s": k / (np.mean(ms) * 1e-3),
           "graph_replay": {"ms_per_step": float(np.mean(g_ms)), "value": atoms / (np.mean(g_ms) * 1e-3)},
           "phase_ms_per_step": {p: v / n for p, v in ph.items()},
           "roofline": {"bound": "alu", "kernel": f"k_moments<float,{L}>", "achieved": ach, "peak": peak_fp32,
                        "unit": "T FP32-pipe lane-instr/s", "frac": ach / peak_fp32, "launch_ms": mom_launch_ms,
                        "traffic": captured_traffic("k_moments_pes_scan_L20.md", ["moments_kernel.cuh", "tcm_internal.h"])},
           "contract_roofline": {"bound": "fp64", "achieved": con, "peak": peak_fp64, "unit": "G FP64 op/s",
                                 "frac": con / peak_fp64, "launch_ms": con_launch_ms,
                                 "algorithmic_fp64_per_energy": contract_fp64_ops(L)},
           "tiling": ({"atoms_per_lane": tuned.best[L][0], "ctas_per_sm": tuned.best[L][1], "kmax": tuned.best[L][2],
                       "chunks": ctx.tcm_ctx_get_chunking_l(L)[1]} if tuned else (fixed or "default"))}
    # B's moments rotated from a cache (Wigner rotation in the contraction kernel) instead of
    # recomputed from its atoms: moments of A and B once, outside the timed steps
    mA = ctx.tcm_moments(A, L, precision=prec)
    mB = ctx.tcm_moments(B, L, precision=prec)
    rc_pb = tcm.pack_batch([tcm.make_system(A, mA.center, mA.radius, moments=mA),
                            tcm.make_system(B, mB.center, mB.radius, moments=mB)], ia, ib, il, s.R0, rotB=s.rotB)
    ctx.tcm_ctx_set_rotate_cached(True)
    r_ms = timer.run(lambda: ctx.tcm_energy_batch_packed(rc_pb, prec, E, st), steps, 3)
    ctx.tcm_ctx_set_rotate_cached(False)
    out["rotate_cached"] = {"ms_per_step": float(np.mean(r_ms)), "energies_per_s": k / (np.mean(r_ms) * 1e-3),
                            "how": "B's cached moments rotated per orientation by Wigner matrices in the contraction "
                                   "kernel (O(L^3)); no atom pass per step"}
    # the same batch in double precision throughout
    ctx.tcm_ctx_set_profiling(True)
    ctx.tcm_ctx_read_profile()
    d_ms = timer.run(lambda: ctx.tcm_energy_batch_packed(pb, tcm.TCM_FP64, E, st), 3, 1)
    ph, la = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    d_mom = ph["moments"] / max(1, la["moments"])
    d_ach = atoms * moment_instr_per_atom(L) / (d_mom * 1e-3) / 1e9
    out["fp64_batched_gpu"] = {"ms_per_step": float(np.mean(d_ms)), "value": atoms / (np.mean(d_ms) * 1e-3),
                               "energies_per_s": k / (np.mean(d_ms) * 1e-3),
                               "moments_roofline": {"bound": "fp64", "achieved": d_ach, "peak": peak_fp64,
                                                    "unit": "G FP64 instr/s", "frac": d_ach / peak_fp64}}
    ctx.close()
    return out


def bench_config3(torch, tcm, synth, stream, prec, calls=3, tune=True):
    """4,096 uneven pairs in one call.  Each timed call is a single call of its shape (graph capture
    on the first call is on): the host planning, the descriptor upload, the capture and the
    kernels are all inside the timed region."""
    from paper_0704_1672_gb300 import autotune
    t0 = time.perf_counter()
    b = synth.uneven_batch()
    t_gen = time.perf_counter() - t0
    T = [(torch.tensor(x, dtype=torch.float32, device="cuda"), None, None) for x in b.systems]
    atoms = int(sum(len(x) for x in b.systems))
    comps = int(sum((int(b.L[i]) + 1) ** 2 * (len(b.systems[b.pair_a[i]]) + len(b.systems[b.pair_b[i]]))
                    for i in range(len(b.L))))
    ctx = tcm.Context(lmax_cap=24, stream=stream)
    tuned = autotune.tune(ctx, T, b.pair_a, b.pair_b, b.L, b.R0, rotB=b.rotB, precision=prec, reps=2,
                          max_items_per_l=256) if tune else None
    E = torch.empty(len(b.L), dtype=torch.float64, device="cuda")
    st = torch.empty(len(b.L), dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(99)
    ctx.tcm_ctx_set_graphs(2)  # capture the launch sequence on the call's first sight of its shape
    pb = tcm.pack_batch(T, b.pair_a, b.pair_b, b.L, b.R0, rotB=b.rotB)  # the system descriptors, marshalled once
    res = []
    for c in range(calls):
        # a fresh set of orientations per call (same pairs and degrees): each call is timed alone,
        # the item array marshalled inside the timed region
        rot = b.rotB if c == 0 else synth.random_rotations(rng, len(b.L))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tw = time.perf_counter()
        e0.record(stream)
        pb.items["rotB"] = rot.reshape(len(b.L), 9)
        ctx.tcm_energy_batch_packed(pb, prec, E, st)
        th = time.perf_counter()  # the call has planned, uploaded and queued its work
        e1.record(stream)
        torch.cuda.synchronize()
        res.append((e0.elapsed_time(e1), (time.perf_counter() - tw) * 1e3, (th - tw) * 1e3))
    ctx.tcm_ctx_set_profiling(True)
    ctx.tcm_ctx_read_profile()
    ctx.tcm_energy_batch_packed(pb, prec, E, st)
    ph, la = ctx.tcm_ctx_read_profile()
    ctx.tcm_ctx_set_profiling(False)
    caps, glaunch = ctx.tcm_ctx_graph_stats()
    ctx.close()
    dev_ms = [r[0] for r in res]
    wall_ms = [r[1] for r in res]
    host_ms = [r[2] for r in res]
    return {"workload": b.name, "pairs": len(b.L), "systems": len(b.systems), "atoms": atoms,
            "atom_moment_components": comps, "calls": calls,
            "call_ms_device": dev_ms, "call_ms_wall": wall_ms, "call_ms_host_queueing": host_ms,
            "value": atoms / (np.median(dev_ms) * 1e-3), "unit": UNIT,
            "energies_per_s": len(b.L) / (np.median(dev_ms) * 1e-3),
            "moment_components_per_s": comps / (np.median(dev_ms) * 1e-3),
            "phase_ms_one_call": ph, "launches_one_call": la, "graph_captures": caps, "graph_launches": glaunch,
            "tiling": ({str(L): list(v) for L, v in tuned.best.items()} if tuned else "default"),
            "tiling_key": "L: [atoms_per_lane, ctas_per_sm, kmax]", "generator_s": t_gen,
            "how": "each call is timed alone (CUDA events around one tcm_energy_batch call, with its host planning, "
                   "descriptor upload and, on a shape's first call, the graph capture); calls 2 and 3 use new "
                   "orientations"}


def bench_serving(torch, tcm, synth, seconds, dev, no_clocks):
    """Serving stream: Poisson arrivals at 2,000 requests/s for `seconds` over 512 resident systems."""
    from paper_0704_1672_gb300 import serve
    stm = synth.serve_stream(seconds=seconds)
    ex = serve.GpuExecutor(stm.systems, device=dev)
    eng = serve.Engine(ex, ex.item_bytes, budget_bytes=4 << 30, max_items=8192, quota=512)
    reqs = serve.make_requests(stm)
    # warm-up on the first requests' shapes (kernel attributes, staging buffers), untimed
    warm = serve.make_requests(stm, seconds=0.05)
    for r in warm:
        r.arrival = 0.0
    serve.Engine(ex, ex.item_bytes, budget_bytes=4 << 30, max_items=8192, quota=512).run_stream(warm)
    atom_moments = sum(r.n * ex.natoms[r.b] for r in reqs)
    clocks = ClockSampler(dev).start() if not no_clocks else None
    m = eng.run_stream(reqs)
    ck = clocks.stop() if clocks else no_clocks()
    m["atom_moments_per_s"] = atom_moments / max(m["seconds"], 1e-12)
    m["workload"] = stm.name
    m["offered_requests_per_s"] = len(reqs) / seconds
    m["clocks"] = ck
    # the plain FP64 per-request path on the first requests of the same stream, and the served
    # results of those requests against it
    sample = serve.make_requests(stm)[:100]
    e_s, a_s = serve.plain_fp64(ex, sample)
    m["plain_fp64_gpu"] = {"energies_per_s": e_s, "atom_moments_per_s": a_s, "requests": len(sample),
                           "how": "one request at a time: tcm_moments (FP64) per side and orientation + tcm_energy"}
    m["served_vs_plain_fp64_energies_per_s"] = m["energies_per_s"] / e_s
    m["accuracy_vs_fp64"] = served_accuracy(ex, eng, tcm, torch, sample[:20])
    return m


def served_accuracy(ex, eng, tcm, torch, sample):
    """|E_served - E_fp64| / |E_fp64| over the items of the sampled requests (served results from the
    engine's completed requests, FP64 from the single-request path)."""
    done = {r.rid: r for r in eng.done}
    ctx = tcm.Context(lmax_cap=24)
    errs = []
    for r in sample:
        d = done.get(r.rid)
        if d is None:
            continue
        da, db = ex.descr[r.a], ex.descr[r.b]
        ma = ctx.tcm_moments(ex.coords[r.a], r.L, precision=tcm.TCM_FP64, center=da.center, radius=da.radius)
        for kk in range(r.n):
            mb = ctx.tcm_moments(ex.coords[r.b], r.L, precision=tcm.TCM_FP64, rot=r.rot[kk], center=db.center,
                                 radius=db.radius)
            e = ctx.tcm_energy(ma, mb, r.R0[kk], r.L)
            errs.append(abs(d.E[kk] - e) / abs(e))
    ctx.close()
    errs = np.array(errs)
    return {"items": len(errs), "median_rel": float(np.median(errs)), "p99_rel": float(np.percentile(errs, 99)),
            "max_rel": float(errs.max()), "fraction_within_1e-6": float((errs <= 1e-6).mean())}


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


def plain_fp64_config4(ctx, tcm, torch, A, B, s, n_orient=8):
    """The plain FP64 GPU path on the headline workload: one request at a time through tcm_moments
    + tcm_energy, no batching; A's moments once, then per orientation B's rotated moments and the
    energy (synchronous), on the first n_orient orientations, extrapolated per step."""
    L = s.L
    qA = torch.empty((L + 1) ** 2, dtype=torch.float64, device="cuda")
    qB = torch.empty((L + 1) ** 2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ma = ctx.tcm_moments(A, L, precision=tcm.TCM_FP64, out=qA)
    torch.cuda.synchronize()
    tA = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i in range(n_orient):
        mb = ctx.tcm_moments(B, L, precision=tcm.TCM_FP64, rot=s.rotB[i], out=qB)
        ctx.tcm_energy(ma, mb, s.R0[i], L)
    torch.cuda.synchronize()
    t_or = (time.perf_counter() - t0) / n_orient
    k = len(s.R0)
    t_step = tA + k * t_or
    atoms = len(s.A) + k * len(s.B)
    return {"value": atoms / t_step, "unit": UNIT, "energies_per_s": k / t_step, "seconds_per_orientation": t_or,
            "seconds_A": tA, "sample": f"A once and {n_orient} orientations, extrapolated to the 10,000-orientation step",
            "how": "per orientation: tcm_moments(B, FP64, rotated) + tcm_energy (synchronous); A once per step"}


def run_only(args):
    """One of the other workloads alone (its record as printed in the full line)."""
    import torch

    from paper_0704_1672_gb300 import autotune, build, synth, tcm
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    smx = sm_max_mhz()
    stream = torch.cuda.current_stream()
    prec = tcm.TCM_MIXED if args.precision == "mixed" else tcm.TCM_FP64
    if args.only == "protein_pes_scan":
        rec = bench_config2(torch, tcm, synth, autotune, Timer(torch, stream), stream, prec,
                            n_sm * FP32_LANES_PER_SM * smx * 1e6 / 1e12, n_sm * FP64_PER_SM_CLK * smx * 1e6 / 1e9,
                            n_sm, smx, steps=args.steps, tune=not args.no_autotune, tiling=args.tiling)
    else:
        rec = bench_config3(torch, tcm, synth, stream, prec, tune=not args.no_autotune)
    print(json.dumps({args.only: rec}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.only:
        run_only(args)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
