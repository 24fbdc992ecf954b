#!/usr/bin/env python3
"""Benchmark of the ms2 MD hot path on GB300: pair interactions per second.

Workload: rigid 3-site water, N = 1000 molecules at 997 kg/m^3 (box 31.07 A),
molecule-centre cut-off 14 A, conducting reaction field, 298 K, leapfrog with
quaternion integration, dt = 2 fs, FP32 site-pair arithmetic with FP64 state
and sums, 1000 NVT steps per job.  One benchmark step = one job: 1000 MD time
steps (partner search + site-pair energies/forces/torques, reduction +
thermostat kick, drift + quaternion rotation + site build, the RDF every 10
steps), run as fused launches of 50 steps.  The job's input state is set
(untimed) before each job; the pairs of a job are counted by replaying it one
step at a time.  Synthetic input: the liquid snapshot
tests/golden/water_N1000.npz (a seeded simple-cubic lattice start with random
orientations and Maxwell-Boltzmann velocities, relaxed by FP64 NVT leapfrog
steps; written by tests/golden/make_snapshots.py).  The GPU arm, the CPU
baseline and the reference arm all start from it.

The L2 cache (129 MB; the whole system is ~0.4 MB) is flushed by writing a
256 MiB buffer between timed jobs, outside the timed interval.  Each job is
timed with CUDA events on the system's stream.  The JSON line also carries the
single MD step per launch, flushed before each (single_step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ms2|reference]

Under torchrun each rank runs an independent replica on its own GPU (the
single-system path does not shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_WATER, RC, SEED = 1000, 14.0, 2
JOB_STEPS = 1000      # NVT steps of one job of the water workload (one bench step)
SINGLE_STEPS = 1000   # flushed single MD steps of the single-step measurement
REF_SAMPLE_STEPS = 5  # the oracle's bounded sample of a job per bench step (reference arm)
SNAPSHOT = os.path.join(ROOT, "tests", "golden", "water_N1000.npz")
RDF_EVERY = 10
# algorithmic FP32 flops per unique water molecule pair (reaction field):
# 9 charge site pairs x 22 + the O-O LJ extra 10 + pair set-up/virial 22
FLOPS_PER_WATER_PAIR = 9 * 22 + 10 + 22
FP32_LANES = 128   # FP32 FMA lanes per SM (Blackwell)


def workload():
    """The benchmark system: 1000 water at 997 kg/m^3, rc = 14 A, in the relaxed
    liquid state of the committed snapshot."""
    import numpy as np
    from paper_1507_07548_gb300 import workloads as W
    wl = W.water_box(N=N_WATER, rc=RC, seed=SEED)
    z = np.load(SNAPSHOT)
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    return wl


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed jobs of %d MD steps" % 1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ms2", choices=["ms2", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle CPU-baseline sample length")
    ap.add_argument("--no-extra", action="store_true", help="skip the Ewald sub-benchmark")
    ap.add_argument("--only", choices=["ewald", "massieu", "thermal", "batch", "serve"], default=None,
                    help="run one sub-benchmark alone and print its JSON object")
    ap.add_argument("--batch-steps", type=int, default=BATCH_STEPS,
                    help="steps of the batch leg (the production length, 10000 in chunks of 100, is opt-in: "
                         "--only batch --batch-steps 10000)")
    ap.add_argument("--batch-kinds", default=None, metavar="K[,K]",
                    help="batch leg: only the systems of these model kinds of the mix (lj, stockmayer, water)")
    ap.add_argument("--uniform-batch", type=int, default=0, metavar="S",
                    help="only time one batch of S copies of the water workload (single steps; the ncu case "
                         "of the multi-system step kernel)")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()

    def summary(self):
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.file.name)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------- CPU baseline
def oracle_rate(seconds, nsteps=None, threads=0):
    """The FP64 oracle (as it stands) stepping the same workload on the host
    cores (all of them, or `threads`); returns (pair interactions/s, steps,
    seconds, threads used)."""
    from oracle import Oracle
    wl = workload()
    o = Oracle.from_workload(wl)
    cores = len(os.sched_getaffinity(0))
    R, q, v, L = wl.R, wl.q, wl.v, wl.Lang
    Oracle.set_threads(threads if threads else cores)
    t0 = time.perf_counter()
    R, q, v, L, th, _ = o.run_leapfrog(R, q, v, L, wl.dt, 1, T0=wl.T)
    t1 = time.perf_counter() - t0
    n = nsteps if nsteps else max(1, int(seconds / max(t1, 1e-6)))
    pairs, dt = 0.0, 0.0
    for _ in range(n):  # only the steps are timed; the pairs are counted outside
        t0 = time.perf_counter()
        R, q, v, L, th, _ = o.run_leapfrog(R, q, v, L, wl.dt, 1, T0=wl.T)
        dt += time.perf_counter() - t0
        pairs += o.partner_counts(R).sum() / 2
    Oracle.set_threads(cores)
    return pairs / dt, n, dt, (threads if threads else cores)


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    from oracle import Oracle
    wl = workload()
    o = Oracle.from_workload(wl)
    cores = len(os.sched_getaffinity(0))
    R, q, v, L = wl.R, wl.q, wl.v, wl.Lang
    # each bench step is a bounded sample of the job: REF_SAMPLE_STEPS MD steps of it
    for _ in range(args.warmup):
        R, q, v, L, _, _ = o.run_leapfrog(R, q, v, L, wl.dt, 1, T0=wl.T)
    R, q, v, L = wl.R, wl.q, wl.v, wl.Lang
    pairs, dt = 0.0, 0.0
    for _ in range(args.steps * REF_SAMPLE_STEPS):
        t0 = time.perf_counter()
        R, q, v, L, _, _ = o.run_leapfrog(R, q, v, L, wl.dt, 1, T0=wl.T)
        dt += time.perf_counter() - t0
        pairs += o.partner_counts(R).sum() / 2
    val = pairs / dt
    line = {"metric": "pair interactions/s", "value": val, "unit": "pair interactions/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "rigid 3-site water N=1000, reaction field, rc=14 A, 298 K, dt=2 fs, leapfrog+quaternion, "
                                   "%d NVT steps per job (one bench step = one job)" % JOB_STEPS,
                       "molecules": N_WATER, "start": "relaxed liquid snapshot (tests/golden/water_N1000.npz)",
                       "parallelism": "host cores (OpenMP owner loop)"},
            "cpu_baseline": {"value": val, "unit": "pair interactions/s", "cores": cores, "kind": "oracle",
                             "sample": "each bench step the first %d MD steps of the job (%d in all)"
                                       % (REF_SAMPLE_STEPS, args.steps * REF_SAMPLE_STEPS)},
            "e2e": {"value": val, "unit": "pair interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
# kernel sources a stored DRAM-traffic figure describes (it is void once they change)
TRAFFIC_SOURCES = {"pair_water_rf": ("k_pair.cu", "pair_engine.cuh", "ms2_internal.cuh"),
                   "step_water_rf_chunk50": ("k_step.cu", "pair_engine.cuh", "integrate_dev.cuh", "grid_dev.cuh",
                                             "ms2_internal.cuh")}


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it still
    describes the current kernel source (matching source hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    csrc = os.path.join(ROOT, "paper_1507_07548_gb300", "csrc")
    try:
        hs = hashlib.sha256()
        for f in TRAFFIC_SOURCES[kernel]:
            hs.update(open(os.path.join(csrc, f), "rb").read())
        h = hs.hexdigest()[:16]
        for line in open(path):
            p = line.split()
            if len(p) >= 3 and p[0] == kernel and p[1] == h:
                return float(p[2])
    except OSError:
        pass
    return None


def combine_ranks(time_ms, work, world):
    """Replicas: the job time is the slowest rank's, the work is summed over ranks
    (gloo collectives on host scalars; the data path has no exchange)."""
    if world <= 1:
        return time_ms, work
    import torch
    import torch.distributed as tdist
    t = torch.tensor([time_ms], dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    w = torch.tensor([work], dtype=torch.float64)
    tdist.all_reduce(w)
    return t.item(), w.item()


def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W

    stream = torch.cuda.Stream()               # a real stream handle shared with the library
    torch.cuda.set_stream(stream)
    wl = workload()
    s = ms2.System.from_workload(wl, stream=stream.cuda_stream)
    s.rdf_setup(min(RC, 0.5 * s.L), 280, every=RDF_EVERY)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    R0, q0, v0, L0 = wl.R, wl.q, wl.v, wl.Lang

    # pairs of one job: the job replayed one step at a time (the same trajectory
    # bit for bit: every launch shape runs the same device functions on the same
    # decomposition), counting each step's partner pairs
    s.set_state(R0, q0, v0, L0)
    job_pairs = 0.0
    for _ in range(JOB_STEPS):
        s.step(1)
        job_pairs += s.energy_terms()["n_pairs"]
    U_replay = s.energy_virial()[0]

    def one_job():
        s.set_state(R0, q0, v0, L0)                  # the job's input into HBM (untimed)
        flush.zero_()                                # evict L2 (outside the timed interval)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(JOB_STEPS)                            # fused launches of 50 steps each
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        one_job()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n0 = ms2.kernel_launches()
    fused = s.fused_step() == 1
    t_job = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            t_job.append(one_job())
    torch.cuda.synchronize()
    launches = ms2.kernel_launches() - n0
    U_job = s.energy_virial()[0]
    tot_ms_max, pairs_all = combine_ranks(sum(t_job), job_pairs * args.steps, world)
    clocks = clk.summary()

    # the flushed single MD step (one fused launch per step), as before the job
    # measurement: its event time and the pair phase inside it
    s.set_state(R0, q0, v0, L0)
    s.enable_timing(True)

    def one_step():
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        tp = s.last_step_times()    # [0] pair kernel (or fused pair phase), [2] the step's kernels
        return e0.elapsed_time(e1), tp[0], tp[2], s.energy_terms()["n_pairs"]

    for _ in range(3):
        one_step()
    t1_step, t1_pair, t1_kern, pairs1 = [], [], [], []
    for _ in range(SINGLE_STEPS):
        a, b, c, d = one_step()
        t1_step.append(a)
        t1_pair.append(b)
        t1_kern.append(c)
        pairs1.append(d)
    s.enable_timing(False)

    # end to end through the public API from host buffers, per job: set_state
    # (H2D of the job's input state through page-locked staging), the job's
    # steps, and the energy read back (D2H)
    e2e_t = 0.0
    for k in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_state(R0, q0, v0, L0)
        s.step(JOB_STEPS)
        U, Wv, T, P = s.energy_virial()
        e2e_t += time.perf_counter() - t0
    h2d = N_WATER * (3 + 4 + 3 + 3) * 8
    d2h = 4 * 8

    extra = {}
    if not args.no_extra and rank == 0:
        extra["ewald_ionic"] = ewald_sub(args, stream)
        extra["massieu"] = massieu_sub(args, stream, flush)
        extra["thermal"] = thermal_sub(args, stream, flush)
        extra["batch"] = batch_sub(args, flush)
        extra["serve"] = serve_sub(args)

    if rank != 0:
        return 0
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak_tflops = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    # dominant kernel: the fused step kernel, JOB_STEPS / 50 launches per job (the
    # first also evaluates the state as set, whose pair phase is not counted)
    per_job = JOB_STEPS // 50 if fused else JOB_STEPS
    kern_ms = statistics.mean(t_job) / per_job
    achieved = FLOPS_PER_WATER_PAIR * job_pairs / per_job / (kern_ms * 1e-3) / 1e12
    traffic = traffic_record("step_water_rf_chunk50" if fused else "pair_water_rf")
    # the flushed single step
    single_ms = statistics.mean(t1_step)
    single_achieved = FLOPS_PER_WATER_PAIR * sum(pairs1) / (sum(t1_kern) * 1e-3) / 1e12
    cpu_val, cpu_n, cpu_dt, cores = oracle_rate(args.cpu_seconds)
    cpu1_val, cpu1_n, cpu1_dt, _ = oracle_rate(max(1.0, args.cpu_seconds / 4), threads=1)
    value = pairs_all / (tot_ms_max * 1e-3)
    line = {
        "metric": "pair interactions/s", "value": value, "unit": "pair interactions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "rigid 3-site water N=1000, reaction field, rc=14 A, 298 K, dt=2 fs, leapfrog+quaternion, "
                               "%d NVT steps per job (one bench step = one job)" % JOB_STEPS,
                   "molecules": N_WATER, "md_steps_per_bench_step": JOB_STEPS,
                   "l2": "flushed between jobs (256 MiB write); a job keeps its state on chip between its steps",
                   "start": "relaxed liquid snapshot (tests/golden/water_N1000.npz), set before each job (untimed)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "state": "FP64 positions/integrator/sums, FP32 site pairs"},
        "molecule_steps_per_s": N_WATER * JOB_STEPS * args.steps * world / (tot_ms_max * 1e-3),
        "site_pair_interactions_per_s": value * 10,
        "pairs_per_job": job_pairs, "replay_matches_job": bool(U_replay == U_job),
        "roofline": {"bound": "alu",
                     "kernel": "k_step<3,1,7,0,RF> (fused MD step, 50 steps per launch)" if fused else "k_pair<3,1,7,0,RF>",
                     "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                     "peak_source": "%d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz max SM clock (unit counts; "
                                    "MEASURED_PEAKS.json has no FP32 figure)" % (sms, sm_max),
                     "kernel_ms": kern_ms,
                     "algorithmic_flops_per_launch": FLOPS_PER_WATER_PAIR * job_pairs / per_job},
        "single_step": {"what": "one MD step per fused launch, L2 flushed before each, CUDA events",
                        "steps": SINGLE_STEPS, "ms_per_step": single_ms,
                        "value": sum(pairs1) / (sum(t1_step) * 1e-3), "unit": "pair interactions/s",
                        "kernel_ms": statistics.mean(t1_kern), "pair_phase_ms": statistics.mean(t1_pair),
                        "achieved_tflops": single_achieved, "frac": single_achieved / peak_tflops},
        "cpu_baseline": {"value": cpu_val, "unit": "pair interactions/s", "cores": cores, "kind": "oracle",
                         "sample": "the first %d MD steps of the job, %.1f s" % (cpu_n, cpu_dt),
                         "single_thread": {"value": cpu1_val, "cores": 1,
                                           "sample": "%d MD steps, %.1f s" % (cpu1_n, cpu1_dt)}},
        "e2e": {"value": job_pairs * args.steps / e2e_t, "unit": "pair interactions/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


BATCH_SYSTEMS, BATCH_STEPS = 512, 200      # many-system mix (production runs: 1e4 steps in chunks of 100)
# the served job stream: 256 jobs with steps 1/100 of production (1e4 - 1e5) and
# arrivals 100x as fast as production's 50/s, so that the offered load in
# molecule-steps/s is the production stream's (several times one GPU's capacity)
SERVE_JOBS, SERVE_RATE, SERVE_STEPS = 256, 5000.0, (100, 1000)
SWEEP_JOBS, SWEEP_STEPS = 48, (100, 1000)   # load-sweep point at ~0.7 of the served capacity
SERVE_RDF_BINS = 100


def batch_sub(args, flush):
    """The same work -- BATCH_SYSTEMS independent systems of the LJ / Stockmayer /
    water mix, --batch-steps steps each (200 by default) -- run one system at a time on one stream
    (each on its best single-system path: the fused step kernel) and as one
    batch (one cooperative multi-system step kernel per model kind).  Host wall time between
    device synchronisations (each run is far longer than a launch), L2 flushed
    before each run."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W
    specs = W.system_mix(BATCH_SYSTEMS, seed=4)
    if args.batch_kinds:  # a sub-mix (profiling one kind's kernel)
        specs = [sp for sp in specs if sp["name"] in args.batch_kinds.split(",")]
    one = torch.cuda.Stream()

    def make(**kw):
        return [ms2.System(sp["models"], sp["counts"], sp["T"], sp["cutoff"], sp["elec"], rho=sp["rho"],
                           seed=sp["seed"], dt=2.0, **kw) for sp in specs]

    plain, batched = make(stream=one.cuda_stream), make()
    steps = args.batch_steps
    work = sum(sp["counts"][0] for sp in specs) * steps
    b = ms2.Batch(batched)
    for s in plain:       # warm-up: one chunk-sized step each, both sets
        s.step(1)
    b.step(1)
    torch.cuda.synchronize()
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in plain:
        s.step(steps)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    fused = sum(s.fused_step() for s in plain)
    b.close()
    for s in plain + batched:
        s.close()
    kinds = {k: sum(1 for sp in specs if sp["name"] == k) for k in W.MIX_STATES}
    return {"workload": "%d independent systems (%s), N ~ U[256, 2048], T ~ U[0.7, 1.3] T0, rho ~ U[0.5, 1.0] rho0; "
                        "%d steps each (production: 1e4)" % (BATCH_SYSTEMS, ", ".join("%d %s" % (v, k) for k, v in
                                                                                      kinds.items()), steps),
            "unit": "molecule-steps/s",
            "plain": {"value": work / t_plain, "seconds": t_plain, "path": "one system at a time, %d of %d fused"
                      % (fused, len(plain))},
            "batched": {"value": work / t_batch, "seconds": t_batch, "path": "multi-system step kernels (one per model kind)"},
            "speedup": t_plain / t_batch}


def run_served(jobs, budget, slots=256):
    """The jobs through the server (ms2_serve_*); arrival times on the server's
    clock.  Returns the results and the span from the first arrival to the last
    result."""
    import paper_1507_07548_gb300.ms2 as ms2
    srv = ms2.Server(budget, slots)
    for j in jobs:
        srv.submit(j["models"], j["counts"], j["T"], j["rho"], j["cutoff"], j["elec"], j["steps"],
                   arrival=j["arrival"], seed=j["seed"], rdf_bins=SERVE_RDF_BINS)
    srv.drain(1800.0)
    res = srv.poll(len(jobs) + 8)
    srv.close()
    span = max(r["t_done"] for r in res) - min(r["t_arrive"] for r in res)
    return res, span


def run_one_at_a_time(jobs):
    """The same jobs, one after the other, each on its own single-system path
    (the fused step kernel where the system allows): create the system as the
    server does, sample the RDF, step, read the averages and g(r).  Returns the
    total time and the latencies of a FIFO queue served this way (each job
    starts at max(its arrival, the previous job's end))."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    total, clock, lat = 0.0, 0.0, []
    for j in jobs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = ms2.System(j["models"], j["counts"], j["T"], j["cutoff"], j["elec"], rho=j["rho"], seed=j["seed"])
        s.rdf_setup(min(s.rc, 0.5 * s.L), SERVE_RDF_BINS, every=10)
        s.reset_averages()
        s.step(j["steps"])
        s.averages()
        s.rdf()
        s.close()
        dt = time.perf_counter() - t0
        total += dt
        clock = max(clock, j["arrival"]) + dt
        lat.append(clock - j["arrival"])
    return total, lat


def serve_sub(args):
    """Serving, two measurements.
    (1) The job stream of the served workload, scaled in time: SERVE_JOBS jobs,
    N ~ U[500, 4000], 80 % the LJ / Stockmayer / water mix and 20 % ionic
    (Ewald), steps 1/100 of the production 10^4 - 10^5 (100 - 1000 in multiples
    of 100) and Poisson arrivals 100 times as fast as the production 50/s, so the
    offered load is the production stream's; energy/pressure averages and g(r)
    out, a 2 GiB admission budget.  The same jobs then run one at a time on the
    single-system path; served / one-at-a-time is the throughput ratio.
    (2) A load sweep point: SWEEP_JOBS jobs of the same kinds arriving at ~0.7 of
    the served capacity just measured, where p50/p99 reflect service time.
    Latency = result on the host minus arrival."""
    import numpy as np
    from paper_1507_07548_gb300 import workloads as W
    jobs = W.job_stream(SERVE_JOBS, SERVE_RATE, seed=5, steps=SERVE_STEPS)
    work = sum(sum(j["counts"]) * j["steps"] for j in jobs)
    res, span = run_served(jobs, 2 << 30)
    lat = np.array([r["t_done"] - r["t_arrive"] for r in res])
    served = work / span
    t_one, lat_one = run_one_at_a_time(jobs)
    one = work / t_one
    stream = {"workload": "%d jobs, N ~ U[500, 4000], 80%% LJ/Stockmayer/water mix + 20%% ionic (Ewald), %d-%d "
                          "steps and Poisson arrivals at %.0f/s (production 1e4-1e5 steps at 50/s, time-scaled by "
                          "1/100: the same offered load), <U>, <P>, g(r) out, 2 GiB budget"
                          % (SERVE_JOBS, SERVE_STEPS[0], SERVE_STEPS[1], SERVE_RATE),
              "completed": int(sum(1 for r in res if r["status"] == 0)), "jobs": len(jobs),
              "served": {"value": served, "seconds": span, "p50_latency_s": float(np.percentile(lat, 50)),
                         "p99_latency_s": float(np.percentile(lat, 99))},
              "one_at_a_time": {"value": one, "seconds": t_one,
                                "p50_latency_s": float(np.percentile(lat_one, 50)),
                                "p99_latency_s": float(np.percentile(lat_one, 99))},
              "served_over_one_at_a_time": served / one, "unit": "molecule-steps/s"}
    probe = W.job_stream(SWEEP_JOBS, 1.0, seed=7, steps=SWEEP_STEPS)
    mean_work = np.mean([sum(j["counts"]) * j["steps"] for j in probe])
    rate = 0.7 * served / mean_work
    sweep = W.job_stream(SWEEP_JOBS, rate, seed=7, steps=SWEEP_STEPS)
    res2, span2 = run_served(sweep, 2 << 30)
    lat2 = np.array([r["t_done"] - r["t_arrive"] for r in res2])
    work2 = sum(sum(j["counts"]) * j["steps"] for j in sweep)
    load = {"workload": "%d jobs of the same kinds, %d-%d steps, Poisson arrivals at %.1f/s (~0.7 of the served "
                        "capacity above)" % (SWEEP_JOBS, SWEEP_STEPS[0], SWEEP_STEPS[1], rate),
            "completed": int(sum(1 for r in res2 if r["status"] == 0)), "jobs": len(sweep),
            "p50_latency_s": float(np.percentile(lat2, 50)), "p99_latency_s": float(np.percentile(lat2, 99)),
            "value": work2 / span2, "unit": "molecule-steps/s"}
    return {"stream": stream, "load_sweep": load,
            # headline figures of the served leg
            "value": served, "unit": "molecule-steps/s", "p50_latency_s": stream["served"]["p50_latency_s"],
            "p99_latency_s": stream["served"]["p99_latency_s"]}


MASSIEU_STEPS = 1000
GK_STEPS = 20000


def massieu_sub(args, stream, flush):
    """The headline water workload with the Massieu moments sampled every step
    (ms2_options.massieu: the pair kernels also sum d2U/dV2), timed the same way:
    L2 flushed, one step per timed interval, CUDA events."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W
    s = ms2.System.from_workload(workload(), stream=stream.cuda_stream, massieu=1)
    s.reset_averages()
    t = []
    for k in range(MASSIEU_STEPS + args.warmup):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            t.append(e0.elapsed_time(e1))
    A, n = s.massieu()
    s.close()
    return {"workload": "rigid 3-site water N=1000, reaction field, rc=14 A, 298 K, Massieu moments every step",
            "ms_per_step": statistics.mean(t), "samples": n,
            "A_r": {k: float(v) for k, v in A.items()},
            "note": "%d samples from the relaxed liquid snapshot: a short run, the values illustrate the output "
                    "rather than converged properties" % n}


def thermal_sub(args, stream, flush):
    """The headline water workload sampling the Green-Kubo heat flux (Eqs. 5-6):
    every step, timed like the headline (L2 flushed, one step per interval), then
    every 5 steps in chunks as a production run would, for lambda."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W
    s = ms2.System.from_workload(workload(), stream=stream.cuda_stream)
    s.heat_setup(every=1, n_lags=8)
    fused = s.fused_step() == 1
    t = []
    for k in range(MASSIEU_STEPS + args.warmup):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            t.append(e0.elapsed_time(e1))
    s.heat_setup(every=5, n_lags=100)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(GK_STEPS)
    e1.record(stream)
    e1.synchronize()
    lam, acf, nsamp = s.thermal_conductivity()
    s.close()
    return {"workload": "rigid 3-site water N=1000, reaction field, rc=14 A, 298 K, heat flux J_q sampled",
            "fused": fused, "ms_per_step_sampled_every_step": statistics.mean(t),
            "ms_per_step_in_chunks": e0.elapsed_time(e1) / GK_STEPS, "steps": GK_STEPS, "extended_step": 5,
            "lags": 100, "samples": nsamp, "lambda_W_per_mK": lam,
            "note": "partial molar enthalpy 0, isokinetic thermostat on (J_q uses the unscaled half-step mean); "
                    "short run: lambda illustrates the output, it is not converged"}


def ewald_sub(args, stream):
    """Ionic solution with Ewald (1000 water + 20 + 20 ions, alpha 0.25, |n| <= 8)."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W
    import numpy as np
    wl = W.ionic_solution(seed=3)
    z = np.load(os.path.join(ROOT, "tests", "golden", "ionic_N1040.npz"))   # relaxed liquid state
    wl.R, wl.q, wl.v, wl.Lang = z["R"], z["q"], z["v"], z["Lang"]
    s = ms2.System.from_workload(wl, stream=stream.cuda_stream)
    s.enable_timing(True)
    fused = s.fused_step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ts, tp, te, pairs = [], [], [], []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        t = s.last_step_times()
        if k >= args.warmup:
            ts.append(e0.elapsed_time(e1))
            tp.append(t[0])
            te.append(t[1])
            pairs.append(s.energy_terms()["n_pairs"])
    # the same system sampling the Green-Kubo current every 5 steps (100 lags = 1 ps),
    # run in chunks as a production run would; the conductivity of so short a
    # run only illustrates the output
    s.enable_timing(False)
    s.conductivity_setup(every=5, n_lags=100)
    nrun = GK_STEPS
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(nrun)
    e1.record(stream)
    e1.synchronize()
    sigma, acf, nsamp = s.conductivity()
    s.close()
    return {"workload": "1000 water + 20 cations + 20 anions, Ewald alpha=0.25/A, |n|<=8 per axis, rc=14 A",
            "value": sum(pairs) / (sum(ts) * 1e-3), "unit": "pair interactions/s",
            "ms_per_step": statistics.mean(ts), "fused": bool(fused),
            # fused: device-timer phases of the step kernel; else the per-phase kernels
            "pair_ms": statistics.mean(tp), "ewald_reciprocal_ms": statistics.mean(te),
            "conductivity": {"ms_per_step_in_chunks": e0.elapsed_time(e1) / nrun, "steps": nrun,
                             "samples": nsamp, "extended_step": 5, "lags": 100, "sigma_S_per_m": sigma,
                             "note": "short run: sigma illustrates the output, it is not converged"}}


def uniform_batch(args):
    """S copies of the headline water system in one batch: `warmup` then `steps`
    single-step batch launches, CUDA events around each, L2 flushed between."""
    import torch
    import paper_1507_07548_gb300.ms2 as ms2
    from paper_1507_07548_gb300 import workloads as W
    wl = workload()
    ss = [ms2.System.from_workload(wl) for _ in range(args.uniform_batch)]
    b = ms2.Batch(ss)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    t = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(1)
        torch.cuda.synchronize()
        if k >= args.warmup:
            t.append(time.perf_counter() - t0)
    pairs = sum(s.energy_terms()["n_pairs"] for s in ss)
    ms = 1e3 * statistics.mean(t)
    print(json.dumps({"workload": "%d x rigid 3-site water N=%d, reaction field, rc=%g A, one batch" % (
        len(ss), N_WATER, RC), "ms_per_step": ms, "pair_interactions_per_s": pairs / (ms * 1e-3),
        "molecule_steps_per_s": len(ss) * N_WATER / (ms * 1e-3), "steps": args.steps}), flush=True)
    b.close()
    return 0


def only_sub(args):
    """One sub-benchmark of the default run, alone (e.g. the ncu case of its kernels)."""
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fn = {"ewald": lambda: ewald_sub(args, stream), "massieu": lambda: massieu_sub(args, stream, flush),
          "thermal": lambda: thermal_sub(args, stream, flush), "batch": lambda: batch_sub(args, flush),
          "serve": lambda: serve_sub(args)}[args.only]
    print(json.dumps({args.only: fn()}), flush=True)
    return 0


def main():
    args = parse()
    if args.uniform_batch > 0:
        return uniform_batch(args)
    if args.only:
        return only_sub(args)
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
    if args.impl == "reference":
        rc = reference_arm(args, rank, world)
    else:
        rc = gpu_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
