#!/usr/bin/env python
"""Benchmark of the direct N-body hot path on GB300.

Workload: Plummer sphere N = 2^20 (seed 3), eps = 1/1024, FP32 pair
arithmetic on double-single positions.  One step = one full-active Hermite
block step on the device (schedule, predict all N, force on all N from all N,
correct + new steps; every particle shares the level 2^-10), i.e. the N^2
sweep with every O(N) stage around it.  Metric: acc+jerk interactions per
second, N (N - 1) per step, also as Gflop/s at 60 flop per interaction and as
a fraction of the FP32 peak.  Energy is measured (full sweeps) before and
after the run.

Beside it, in the same JSON line: the force kernel's roofline (CUDA events
around each force launch on the library's stream), isolated sweeps with
n_active in {1, 256, 4096, 65536, N}, the all-FP64 kernel on the same sweep,
an end-to-end figure through the host-buffer API, the CPU oracle on a bounded
sample of the same workload, and SM clocks sampled during the timed region.

  python bench.py [--gpus N --steps K --warmup W]       # this library
  python bench.py --impl reference [...]                # the CPU oracle
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "acc+jerk interactions/s & % FP32 peak, FP32-DS vs FP64 GPU, at |ΔE/E|≤1e-6"
UNIT = "interactions/s"
FLOP_PER_INTERACTION = 60          # eta_fe of the paper (Section 5)
N_DEFAULT = 1 << 20
EPS = 1.0 / 1024
SEED = 3
LEVEL = 10                         # shared step 2^-10
SWEEP_LADDER = [1, 256, 4096, 65536]
ABOVE_L2_N = 1 << 22               # small-block sweeps with j records larger than the L2
ABOVE_L2_LADDER = [1, 4, 32]
FP64_SAMPLE = 4096
ACCURACY_SAMPLE_FULL = 128         # sampled i of the headline accuracy check
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128
MAX_SM_MHZ_FALLBACK = 2070.0
J_RECORD_BYTES = 48                # DS j record: three float4
SWEEP_HBM_MAX_ACTIVE = 2           # sweeps this small are bound by the j-record stream
HBM_GBS_FALLBACK = 6800.0          # earlier GB300 copy measurement, when no measured file exists


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mine", choices=["mine", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--no-extras", action="store_true", help="skip ladder, FP64 arm, e2e, CPU baseline")
    p.add_argument("--configs", default="1,2,3,4,5",
                   help="default workload: the configurations run after the headline (empty: none)")
    p.add_argument("--workload", default="full_active_step",
                   choices=["full_active_step", "blockstep", "adjoint", "ensemble", "replay", "summation",
                            "sweep"],
                   help="blockstep: individual block steps of a Plummer run (Section 2 step loop)")
    p.add_argument("--t-end", type=float, default=0.25, help="blockstep: end time (multiple of dt_max)")
    p.add_argument("--eps", type=float, default=None, help="blockstep: softening (default 1/256)")
    p.add_argument("--seed", type=int, default=None)
    p.add_argument("--precision", default="ds", choices=["ds", "fp64", "both"])
    p.add_argument("--fd-coords", type=int, default=32, help="adjoint: coordinates checked by FP64 FD")
    p.add_argument("--clusters", type=int, default=4096, help="ensemble: number of clusters")
    p.add_argument("--n-max", type=int, default=524288, help="replay: largest N of the ladder")
    p.add_argument("--baseline-sample", type=int, default=32,
                   help="ensemble: clusters timed one by one through the single-system path")
    p.add_argument("--ens-config", default="",
                   help="ensemble: 'threads,gmax' instead of the autotuner (e.g. for a profiler run, "
                        "under which the tuner's timings are distorted)")
    p.add_argument("--oracle-outliers", type=int, default=0,
                   help="ensemble: re-run this many worst clusters (<= 512 bodies) with the oracle")
    p.add_argument("--oracle-n", type=int, default=1024, help="adjoint: size of the CPU FP64 comparison")
    p.add_argument("--cpu-budget", type=float, default=20.0,
                   help="blockstep: seconds of the oracle's integrator timed beside the GPU run")
    p.add_argument("--n-active", default="1,96,256,4096",
                   help="sweep: comma-separated block sizes, each against all N j")
    p.add_argument("--sample-errors", type=int, default=0,
                   help="blockstep: check this many sampled i against the oracle at each of 16 checkpoints")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu_index = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)), "samples": len(sm), "reasons": sorted(reasons)}


def nvsmi_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [q.strip() for q in vis.split(",") if q.strip()]
    if ids and all(q.isdigit() for q in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------

def max_over_ranks(x, device):
    """Maximum of a per-rank float over the process group (x itself alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step, elapsed_max):
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * steps * units_per_step / elapsed_max


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return HBM_GBS_FALLBACK


def fp32_peak_tflops(sms, mhz):
    """FP32 FMA peak: 128 lanes per SM, 2 flop per FMA."""
    return 2.0 * FP32_LANES_PER_SM * sms * mhz * 1e6 / 1e12


FORCE_SOURCES = ("k_force.cu", "nb_device.cuh", "nb_internal.cuh")
FIXED_SOURCES = ("k_sum.cu", "nb_device.cuh", "nb_internal.cuh")


def force_sources_sha256(sources=FORCE_SOURCES):
    """sha256 over a kernel's sources, concatenated in the order given."""
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_cs_0702135_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def force_traffic_per_launch(n, profile="k_force_ipar_ds.md", sources=FORCE_SOURCES):
    """DRAM bytes per full-N force launch from the committed ncu summary, or
    None when the kernel's sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"force sources sha256[^:]*:\s*([0-9a-f]{64})", text)
    caps = {int(a): float(b) for a, b in
            re.findall(r"dram bytes per launch at N=(\d+):\s*([0-9.eE+]+)", text)}
    if not mh or not caps:
        return None
    if force_sources_sha256(sources) != mh.group(1):
        return None
    if n in caps:
        return caps[n]
    # Otherwise the largest capture, scaled linearly: with the j records
    # resident in L2 and a uniform slice plan the traffic is O(N) (records,
    # block outputs).
    n_cap = max(caps)
    return caps[n_cap] * n / n_cap


def cpu_oracle_rate(m, x, v, eps, budget_s=10.0, seed=SEED, summation=0):
    """Oracle direct-sum force (OpenMP over i) on a growing sample of active i
    against all N j until one timing takes at least budget_s seconds
    (summation > 0: the oracle's summation variant of that number)."""
    import oracle
    from synth import sample_active
    threads = os.cpu_count() or 1
    oracle.lib()
    n = m.shape[0]
    na = 64
    while True:
        idx = sample_active(n, na, seed + na)
        t0 = time.perf_counter()
        if summation:
            oracle.force_summed(m, x, v, eps, idx, mode=summation, nthreads=threads)
        else:
            oracle.force(m, x, v, eps, idx, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt >= budget_s or na >= n:
            break
        na = min(n, max(na * 2, int(na * budget_s / max(dt, 1e-3) * 1.1)))
    return na * (n - 1) / dt, threads, na, dt


def run_reference(args):
    """The oracle as it stands, on the host cores, on this workload's metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from synth import plummer, sample_active
    n = args.n
    m, x, v = plummer(n, SEED)
    threads = os.cpu_count() or 1
    oracle.lib()
    na = max(1, min(n, 256 * max(1, threads // 16)))
    idx = [sample_active(n, na, SEED + s) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        oracle.force(m, x, v, EPS, idx[s], nthreads=threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.force(m, x, v, EPS, idx[args.warmup + s], nthreads=threads)
    el = time.perf_counter() - t0
    rate = args.steps * na * (n - 1) / el
    sample = ("oracle direct-sum force, %d of the %d active i per step against all N j "
              "(the full-active step's N^2 sweep, sampled); O(N) predict/correct not timed" % (na, n))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "plummer_N%d_eps1/1024_full_active_block_step" % n, "N": n,
                       "eps": EPS, "seed": SEED},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": rate,
                             "unit": UNIT},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_mine(args):
    import torch
    import paper_cs_0702135_gb300 as nb
    from synth import plummer, sample_active

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    # A stream of our own: the library runs on it, and the events and the L2
    # flush below are recorded on it too.
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    n = args.n
    inter_per_step = n * (n - 1)

    m, x, v = plummer(n, SEED + rank)      # replicas: one independent sphere per rank
    ctx = nb.Context(m, x, v, EPS, level_fixed=LEVEL, stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    e0 = sum(ctx.nb_energy())

    for _ in range(args.warmup):
        flush.zero_()
        ctx.nb_step(wait=False)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(nvsmi_index(local))
    ctx.nb_get_stats(reset=True)
    ctx.nb_set_profiling(True)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.zero_()                         # L2 flush between steps
        ctx.nb_step(wait=False)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    stats = ctx.nb_get_stats(reset=True)
    ctx.nb_set_profiling(False)
    if world > 1:
        elapsed = max_over_ranks(elapsed, dev)
        torch.distributed.barrier()
    e1 = sum(ctx.nb_energy())
    value = whole_job_rate(world, args.steps, inter_per_step, elapsed)

    force_s = stats["force_ms"] / 1e3 / max(1, stats["force_launches"])
    peak = fp32_peak_tflops(sms, MAX_SM_MHZ_FALLBACK)
    achieved = FLOP_PER_INTERACTION * inter_per_step / force_s / 1e12
    traffic = force_traffic_per_launch(n)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_force_ipar_ds (full-N launch inside the step)",
                "peak_note": "FP32 FMA peak 2 x 128 lanes x %d SMs x 2070 MHz (max SM clock)" % sms}
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / fp32_peak_tflops(sms, clocks["sm_mhz"])

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(args, nb, ctx, m, x, v, stream, dev, torch, sample_active)
        if world == 1 and args.configs:
            extras["configs"] = run_configs(args, nb, torch, stream)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plummer_N%d_eps1/1024_full_active_block_step" % n, "N": n,
                   "eps": EPS, "seed": SEED, "n_active": n, "shared_level": LEVEL,
                   "precision": "FP32 pair terms on double-single positions, FP64 predictor/corrector",
                   "l2": "inputs larger than L2 (~270 MB touched per step) and a 256 MiB memset "
                         "between steps inside the timed region",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gflops": value * FLOP_PER_INTERACTION / 1e9,
        "pct_fp32_peak": 100.0 * value * FLOP_PER_INTERACTION / 1e12 / peak,
        "energy": {"rel_err": abs(e1 - e0) / abs(e0), "steps": args.warmup + args.steps,
                   "dt": 2.0 ** -LEVEL},
        "roofline": roofline,
        "gpu_launches": stats["kernel_launches"],
        "clocks": clocks,
        "device": {"name": props.name, "sms": sms},
    }
    line.update(extras)
    ctx.nb_free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def time_sweeps(ctx, n, nas, dev, torch, sample_active, flush):
    """Isolated force sweeps: for each n_active, that many i (uniform without
    replacement, seed SEED + n_active) against all n j; 5 warm-ups, then the
    median of 20 repetitions (3 for the full sweep), each timed with CUDA
    events around the force kernels, with a memset larger than L2 before each
    (outside the events) so that the j records come from HBM."""
    ladder = {}
    for na in nas:
        idx = torch.from_numpy(sample_active(n, na, SEED + na)).to(dev)
        acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
        jerk = torch.empty_like(acc)
        pot = torch.empty(na, dtype=torch.float64, device=dev)
        reps = 3 if na == n else 20
        for _ in range(5):
            ctx.nb_force_dev(idx, na, acc, jerk, pot)
        ctx.nb_set_profiling(True)
        times, launches = [], 0
        t0 = time.perf_counter()
        for _ in range(reps):
            # (the stats reset synchronises: it goes first, so the flush is
            # still running when the force is enqueued and no host gap falls
            # between the CUDA events around the force kernels)
            ctx.nb_get_stats(reset=True)
            flush.zero_()
            ctx.nb_force_dev(idx, na, acc, jerk, pot)
            st = ctx.nb_get_stats(reset=True)
            times.append(st["force_ms"] / 1e3 / max(1, st["force_launches"]))
            launches += st["kernel_launches"]
        torch.cuda.synchronize(dev)
        call_s = (time.perf_counter() - t0) / reps
        ctx.nb_set_profiling(False)
        fs = float(np.median(times))
        # every sweep streams the 48-byte j records once: for a handful of
        # active i that is the bound
        jbytes = J_RECORD_BYTES * n
        ladder[str(na)] = {"force_us": fs * 1e6, "force_us_mean": float(np.mean(times)) * 1e6,
                           "repetitions": reps, "wall_us_per_rep": call_s * 1e6,
                           "kernel_launches": launches,
                           "interactions_per_s": na * (n - 1) / fs,
                           "gflops": FLOP_PER_INTERACTION * na * (n - 1) / fs / 1e9,
                           "j_record_gbs": jbytes / fs / 1e9,
                           "j_record_hbm_frac": jbytes / fs / 1e9 / hbm_peak_gbs()}
    return ladder


def time_sweeps_above_l2(nb, torch, stream, dev, sample_active, n=ABOVE_L2_N):
    """Small-block sweeps whose j records do not fit the L2: Plummer N = 2^22
    (seed 3), eps = 1/1024, 48 B x N = 201 MB of records against the 129 MB
    L2, so no flush is needed (and none leaves dirty lines behind); 5 warm-ups,
    then the median of 20 launches timed with CUDA events around the force
    kernels."""
    from synth import plummer
    m, x, v = plummer(n, SEED)
    c = nb.Context(m, x, v, EPS, flags=nb.NB_INIT_NO_FORCE, stream=stream.cuda_stream)
    out = {}
    try:
        for na in ABOVE_L2_LADDER:
            idx = torch.from_numpy(sample_active(n, na, SEED + na)).to(dev)
            acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
            jerk, pot = torch.empty_like(acc), torch.empty(na, dtype=torch.float64, device=dev)
            for _ in range(5):
                c.nb_force_dev(idx, na, acc, jerk, pot)
            c.nb_set_profiling(True)
            c.nb_get_stats(reset=True)
            times = []
            for _ in range(20):
                c.nb_force_dev(idx, na, acc, jerk, pot)
                st = c.nb_get_stats(reset=True)
                times.append(st["force_ms"] / 1e3 / max(1, st["force_launches"]))
            c.nb_set_profiling(False)
            fs = float(np.median(times))
            jbytes = J_RECORD_BYTES * n
            out[str(na)] = {"force_us": fs * 1e6, "j_record_gbs": jbytes / fs / 1e9,
                            "j_record_hbm_frac": jbytes / fs / 1e9 / hbm_peak_gbs(),
                            "interactions_per_s": na * (n - 1) / fs}
    finally:
        c.nb_free()
    return {"N": n, "records_mb": J_RECORD_BYTES * n / 1e6, "flush": "none (records exceed L2)",
            "sweeps": out}


def run_extras(args, nb, ctx, m, x, v, stream, dev, torch, sample_active):
    n = args.n
    out = {}
    # Isolated sweeps: n_active i (uniform without replacement) against all N j.
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ladder = time_sweeps(ctx, n, [na for na in SWEEP_LADDER + [n] if na <= n], dev, torch,
                         sample_active, flush)
    out["sweeps"] = ladder
    out["sweeps_above_l2"] = time_sweeps_above_l2(nb, torch, stream, dev, sample_active)

    # The all-FP64 kernel on the same sweep (FP64_SAMPLE active i against all N).
    na = min(FP64_SAMPLE, n)
    c64 = nb.Context(m, x, v, EPS, precision=nb.NB_FP64, flags=nb.NB_INIT_NO_FORCE,
                     stream=stream.cuda_stream)
    idx = torch.from_numpy(sample_active(n, na, SEED + na)).to(dev)
    acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
    c64.nb_force_dev(idx, na, acc, None, None)
    c64.nb_get_stats(reset=True)
    c64.nb_set_profiling(True)
    for _ in range(3):
        c64.nb_force_dev(idx, na, acc, None, None)
    st = c64.nb_get_stats(reset=True)
    c64.nb_set_profiling(False)
    # Accuracy of both GPU forms against the FP64 oracle on sampled particles
    # of the initial state (per-particle metric of the parity tests).
    import oracle
    ia = sample_active(n, min(ACCURACY_SAMPLE_FULL, n), SEED + 29)
    ref = oracle.force(m, x, v, EPS, ia, nthreads=os.cpu_count() or 1)
    sa, sk = pair_magnitude_sums(m, x, v, EPS, ia, chunk=8)
    cds = nb.Context(m, x, v, EPS, flags=nb.NB_INIT_NO_FORCE, stream=stream.cuda_stream)
    acc_rows = {}
    for name, c in (("ds", cds), ("fp64_gpu", c64)):
        e = force_error_stats(c.nb_force(ia), ref, sa, sk)
        acc_rows[name] = {"max_err_acc": e[0], "max_err_jerk": e[1], "max_err_pot": e[2],
                          "p99_raw_rel_acc": e[3]}
    # The timed sweep itself (all n i active): sampled outputs of one full-n
    # force against the oracle, half of them from the last eighth of the
    # particles, where the plan's sliced remainder lies (its first i-blocks
    # run whole).
    rng = np.random.default_rng(SEED + 31)
    cut = n - n // 8
    half = min(ACCURACY_SAMPLE_FULL // 2, cut, n - cut)
    pick = np.sort(np.concatenate([rng.choice(cut, half, replace=False),
                                   cut + rng.choice(n - cut, half, replace=False)])).astype(np.int32)
    full = cds.nb_force(np.arange(n, dtype=np.int32))
    ref_f = oracle.force(m, x, v, EPS, pick, nthreads=os.cpu_count() or 1)
    fa_, fk_ = pair_magnitude_sums(m, x, v, EPS, pick, chunk=8)
    e = force_error_stats(tuple(g[pick] for g in full), ref_f, fa_, fk_)
    acc_rows["ds_full_sweep"] = {"max_err_acc": e[0], "max_err_jerk": e[1], "max_err_pot": e[2],
                                 "p99_raw_rel_acc": e[3],
                                 "sample": "%d of the %d outputs of one all-active sweep, %d of them "
                                           "from the last eighth" % (len(pick), n, half)}
    del full
    cds.nb_free()
    c64.nb_free()
    acc_rows["sample"] = ("%d i drawn uniformly (seed %d) against all %d j at t = 0; err = |d| / "
                          "max(|ref|, S/10), S the sum of pair magnitudes (pot: relative)"
                          % (len(ia), SEED + 29, n))
    acc_rows["tolerance"] = {"acc": 2e-6, "jerk": 1e-5, "pot": 2e-6}
    out["accuracy_vs_oracle"] = acc_rows
    fs64 = st["force_ms"] / 1e3 / max(1, st["force_launches"])
    r64 = na * (n - 1) / fs64
    rds = ladder[str(na)]["interactions_per_s"] if str(na) in ladder else None
    out["fp64_gpu"] = {"value": r64, "unit": UNIT, "sample": "%d active i against all %d j" % (na, n),
                       "ds_over_fp64": (rds / r64) if rds else None}

    out["e2e"] = e2e_host_api(ctx, nb, n, max(2, min(args.steps, 3)), torch, dev)

    # The CPU oracle on a bounded sample of the same workload.
    if int(os.environ.get("WORLD_SIZE", "1")) == 1:
        rate, threads, na_s, secs = cpu_oracle_rate(m, x, v, EPS)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "oracle direct-sum force (FP64, OpenMP) on %d of the %d "
                                         "active i against all j, %.1f s" % (na_s, n, secs)}
    return out


CONFIG_NAMES = {
    1: "plummer_N1024_eps1/256_t0-1_blockstep",
    2: "plummer_N65536_eps1/256_t0-0.25_blockstep",
    3: "plummer_N1048576_eps1/1024_t0-1/16_blockstep",
    4: "adjoint_plummer_N16384_eps1/256_dt1/1024_steps256_ckpt16",
    5: "ensemble_4096_plummer_salpeter_N32-4096_eps1/256_t1",
}


def run_configs(args, nb, torch, stream):
    """Every workload configuration of the benchmark suite, each with its own
    clock (wall seconds of the entry), after the headline measurement:
    1. N = 1024 to t = 1, DS and FP64 GPU, the oracle's whole run beside it;
    2. N = 65536 to t = 1/4, DS and FP64 GPU, block-size histogram, sampled
       force errors against the oracle at 16 checkpoints, energies against the
       oracle's pair sums;
    3. N = 2^20 (eps = 1/1024) to t = 1/16, DS;
    4. the differentiable run (adjoint, FD and oracle checks);
    5. the batched ensemble of 4096 clusters, its worst clusters re-run by the
       oracle."""
    out = {}
    want = sorted({int(c) for c in args.configs.split(",") if c.strip()})
    for c in want:
        t0 = time.perf_counter()
        if c == 1:
            r = blockstep_config(nb, torch, stream, 1024, 1, 1.0 / 256, 1.0, [nb.NB_DS, nb.NB_FP64],
                                 cpu_budget=20.0, energy_vs_oracle=True)
        elif c == 2:
            r = blockstep_config(nb, torch, stream, 65536, 2, 1.0 / 256, 0.25, [nb.NB_DS, nb.NB_FP64],
                                 sample_errors=1024, cpu_budget=10.0, energy_vs_oracle=True)
        elif c == 3:
            r = blockstep_config(nb, torch, stream, 1 << 20, 3, 1.0 / 1024, 1.0 / 16, [nb.NB_DS],
                                 block_sizes=False, cpu_budget=10.0)
            ds = r["ds"]
            peak = fp32_peak_tflops(torch.cuda.get_device_properties(0).multi_processor_count,
                                    MAX_SM_MHZ_FALLBACK)
            ds["pct_fp32_peak"] = 100.0 * ds["gflops"] / 1e3 / peak
        elif c == 4:
            r = adjoint_config(nb, torch, 16384, 32, 1024)
        elif c == 5:
            r = ensemble_config(nb, torch, 4096, 32, oracle_outliers=5, oracle_n_max=512)
        else:
            continue
        r["wall_s"] = time.perf_counter() - t0
        out["%d_%s" % (c, CONFIG_NAMES[c])] = r
    return out


def e2e_host_api(ctx, nb, n, k_e2e, torch, dev):
    """End to end through the host-buffer API: per full-active step nb_predict,
    nb_force with pinned host index/output arrays, nb_correct; the copies are
    inside the timed region."""
    st0 = ctx.nb_get_state()
    t_cur = int(st0["t"].max())
    dt = 1 << (40 - LEVEL)
    idx_h = torch.arange(n, dtype=torch.int32).pin_memory().numpy()
    acc_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    jerk_h = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    pot_h = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for s in range(k_e2e):
        t_cur += dt
        ctx.nb_predict(t_cur / nb.TICKS_PER_UNIT)
        nb.nb_force_into(ctx.ctx, idx_h, acc_h, jerk_h, pot_h)
        ctx.nb_correct(idx_h, t_cur / nb.TICKS_PER_UNIT)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    return {"value": k_e2e * n * (n - 1) / el, "unit": UNIT,
            "h2d_bytes_per_step": 2 * 4 * n, "d2h_bytes_per_step": (3 + 3 + 1) * 8 * n,
            "steps": k_e2e, "api": "nb_predict + nb_force (host arrays) + nb_correct"}


def blockstep_config(nb, torch, stream, n, seed, eps, t_end, precisions, block_sizes=True,
                     sample_errors=0, cpu_budget=20.0, energy_vs_oracle=False):
    """A Plummer run with individual block steps on the device (nb_run, graph
    replay or the persistent launch): interactions/s over the whole run,
    |dE/E|, and for the DS path the block-size distribution (from a
    step-by-step replay of the same run) and, with sample_errors > 0, the
    force on that many sampled particles at 16 checkpoints against the FP64
    oracle.  Beside it the oracle's own integrator on the host cores."""
    from synth import plummer
    level_min = 3
    while (2.0 ** -level_min) > t_end or (t_end / 2.0 ** -level_min) % 1:
        level_min += 1
    m, x, v = plummer(n, seed)
    out = {"workload": "blockstep_plummer_N%d_eps%g_t%g" % (n, eps, t_end), "N": n, "eps": eps,
           "seed": seed, "t_end": t_end, "level_min": level_min, "eta": 0.01}
    for prec in precisions:
        name = "ds" if prec == nb.NB_DS else "fp64"
        ctx = nb.Context(m, x, v, eps, precision=prec, level_min=level_min, stream=stream.cuda_stream)
        e0 = sum(ctx.nb_energy())
        st0 = ctx.nb_get_state()
        ctx.nb_get_stats(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, inter = ctx.nb_run(t_end)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        launches = ctx.nb_get_stats(reset=True)["kernel_launches"]
        e1 = sum(ctx.nb_energy())
        res = {"steps": steps, "interactions": inter, "seconds": el, "interactions_per_s": inter / el,
               "gflops": 60 * inter / el / 1e9, "us_per_step": 1e6 * el / max(1, steps),
               "energy_t0": e0, "energy_t_end": e1,
               "energy_rel_err": abs(e1 - e0) / abs(e0), "kernel_launches": launches}
        if energy_vs_oracle:
            # the GPU's energy (a full force sweep in the context's precision)
            # against the oracle's FP64 pair sum of the same state
            import oracle
            thr = os.cpu_count() or 1
            sT = ctx.nb_get_state()
            o0 = sum(oracle.energy(m, st0["x"], st0["v"], eps, thr))
            o1 = sum(oracle.energy(m, sT["x"], sT["v"], eps, thr))
            res["energy_vs_oracle_rel"] = {"t0": abs(e0 - o0) / abs(o0), "t_end": abs(e1 - o1) / abs(o1)}
        if prec == nb.NB_DS and (block_sizes or sample_errors):
            # replay the same run step by step for the block sizes (and sampled errors)
            ctx.nb_set_state(st0["x"], st0["v"], st0["a"], st0["k"], st0["t"], st0["level"])
            sizes = []
            checks = set(np.linspace(0, steps - 1, 16).astype(int).tolist()) if sample_errors else set()
            errs = []
            for s_ in range(steps):
                if s_ in checks:
                    errs.append(sampled_force_errors(ctx, nb, m, eps, sample_errors, seed + s_))
                tb, na = ctx.nb_step()
                sizes.append(na)
            sizes = np.array(sizes)
            edges = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384, 32768,
                     65536, 131072, 262144, 524288, 1048576, 2097152]
            hist, _ = np.histogram(sizes, bins=edges + [10 ** 12])
            res["n_active"] = {"mean": float(sizes.mean()), "median": float(np.median(sizes)),
                               "max": int(sizes.max()), "min": int(sizes.min()),
                               "hist_log2_bins": {str(e): int(h) for e, h in zip(edges, hist) if h},
                               "paper_fit_n_block": 0.20 * n ** 0.81,
                               "paper_fit_steps": 247 * n ** 0.35 * t_end}
            if errs:
                res["sampled_errors"] = {
                    "checkpoints": len(errs), "per_checkpoint_i": sample_errors,
                    "metric": "|d|/max(|ref|, S/10) per particle, S = sum of pair magnitudes; pot relative",
                    "max_err_acc": max(e[0] for e in errs), "max_err_jerk": max(e[1] for e in errs),
                    "max_err_pot": max(e[2] for e in errs), "p99_raw_rel_acc": max(e[3] for e in errs),
                    "within_tolerance": bool(max(e[0] for e in errs) <= 2e-6
                                             and max(e[1] for e in errs) <= 1e-5
                                             and max(e[2] for e in errs) <= 2e-6)}
        out[name] = res
        ctx.nb_free()
    if "ds" in out and "fp64" in out:
        out["ds_over_fp64"] = out["ds"]["interactions_per_s"] / out["fp64"]["interactions_per_s"]
    if cpu_budget > 0:
        out["cpu_baseline"] = oracle_blockstep_rate(m, x, v, eps, level_min, t_end,
                                                    out.get("ds", out.get("fp64")), cpu_budget)
    return out


def run_blockstep(args):
    import torch
    import paper_cs_0702135_gb300 as nb
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    precs = {"ds": [nb.NB_DS], "fp64": [nb.NB_FP64], "both": [nb.NB_DS, nb.NB_FP64]}[args.precision]
    out = blockstep_config(nb, torch, stream, args.n,
                           args.seed if args.seed is not None else 2,
                           args.eps if args.eps is not None else 1.0 / 256, args.t_end, precs,
                           sample_errors=args.sample_errors,
                           cpu_budget=0.0 if args.no_extras else args.cpu_budget)
    print(json.dumps(out), flush=True)


def oracle_blockstep_rate(m, x, v, eps, level_min, t_end, gpu, budget_s):
    """The oracle's FP64 integrator (OpenMP force on all host cores) from the
    same initial conditions: the whole run when it ends within budget_s, else
    its first block steps until budget_s has passed; interactions/s over those
    steps and, for a partial run, the full run's time projected from the GPU
    run's interaction count at that rate (stated)."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.lib()
    n = m.shape[0]
    if float(n) * n > 5e8 * budget_s:
        # the integrator's start-up sweep alone (n^2 FP64 pairs) would exceed the
        # budget: time the oracle's force on a sample of the particles instead
        rate, thr, na_s, secs = cpu_oracle_rate(m, x, v, eps, budget_s=budget_s / 2)
        res = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "whole_run": False,
               "sample": "the oracle's FP64 force (OpenMP) on %d of the %d particles against all j, "
                         "%.1f s (its integrator's start-up sweep alone would exceed the %.0f s "
                         "budget); whole run projected from the GPU run's interaction count"
                         % (na_s, n, secs, budget_s)}
        if gpu and rate > 0:
            res["projected_whole_run_s"] = gpu["interactions"] / rate
            res["gpu_over_oracle"] = gpu["interactions_per_s"] / rate
        return res
    t0 = time.perf_counter()
    orc = oracle.Integrator(m, x, v, eps, kmin=level_min, nthreads=threads)
    init_s = time.perf_counter() - t0
    e0 = orc.energy() if n <= 16384 else None
    t_end_ticks = int(round(t_end * oracle.TICKS_PER_UNIT))
    steps, inter, done = 0, 0, False
    t0 = time.perf_counter()
    while True:                       # at least one step, then until the budget is spent
        tn, act = orc.step(t_end_ticks)
        if len(act) == 0 or tn > t_end_ticks:
            done = True
            break
        steps += 1
        inter += len(act) * (n - 1)
        if tn == t_end_ticks and int(orc.t.min()) == t_end_ticks:
            done = True
            break
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    rate = inter / el if el > 0 else 0.0
    res = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "steps": steps,
           "seconds": el, "startup_sweep_s": init_s, "whole_run": done}
    if done:
        res["sample"] = "the oracle's whole run (%d block steps, %.1f s after a %.1f s start-up sweep)" % (
            steps, el, init_s)
        if e0 is not None:
            res["energy_rel_err"] = abs(orc.energy() - e0) / abs(e0)
        if gpu:
            res["gpu_steps_over_oracle_steps"] = gpu["steps"] / max(1, steps)
    else:
        proj = gpu["interactions"] / rate if rate > 0 else None
        res["sample"] = ("the oracle's first %d block steps of the same run (%.1f s; the GPU run took "
                         "%d); whole run projected at %.0f s from the GPU run's interaction count"
                         % (steps, el, gpu["steps"], proj or float("nan")))
        res["projected_whole_run_s"] = proj
    if gpu and rate > 0:
        res["gpu_over_oracle"] = gpu["interactions_per_s"] / rate
    return res


def pair_magnitude_sums(m, x, v, eps, idx, chunk=16):
    """Per listed i: S_a = sum_j |m_j dx / r^3| and S_k = sum_j |jerk_ij| (j != i),
    the scales of the per-particle force error metric; chunked over i."""
    sa = np.empty(len(idx))
    sk = np.empty(len(idx))
    for s0 in range(0, len(idx), chunk):
        ii = np.asarray(idx[s0:s0 + chunk])
        d = x[None, :, :] - x[ii, None, :]
        w = v[None, :, :] - v[ii, None, :]
        r2 = np.einsum("ijk,ijk->ij", d, d) + eps * eps
        rv = np.einsum("ijk,ijk->ij", d, w)
        with np.errstate(divide="ignore", invalid="ignore"):
            r3 = r2 ** -1.5
            fa = m[None, :] * np.sqrt(r2 - eps * eps) * r3
            kk = m[None, :, None] * (w * r3[..., None] - 3 * (rv * r3 / r2)[..., None] * d)
            fk = np.linalg.norm(kk, axis=2)
        rows = np.arange(len(ii))
        fa[rows, ii] = 0.0
        fk[rows, ii] = 0.0
        sa[s0:s0 + len(ii)] = np.nansum(fa, axis=1)
        sk[s0:s0 + len(ii)] = np.nansum(fk, axis=1)
    return sa, sk


def force_error_stats(got, ref, sa, sk):
    """(max err_a, max err_k, max err_pot, p99 raw |da|/|a|): err_a = |da| /
    max(|a|, S_a/10), the same for the jerk; the potential's plain relative error."""
    ea = np.linalg.norm(got[0] - ref[0], axis=1) / np.maximum(np.linalg.norm(ref[0], axis=1), sa / 10)
    ek = np.linalg.norm(got[1] - ref[1], axis=1) / np.maximum(np.linalg.norm(ref[1], axis=1), sk / 10)
    ep = np.abs(got[2] - ref[2]) / np.abs(ref[2])
    raw = np.linalg.norm(got[0] - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1)
    return float(ea.max()), float(ek.max()), float(ep.max()), float(np.percentile(raw, 99))


def sampled_force_errors(ctx, nb, m, eps, k, seed):
    """Force on k sampled particles at the current (synchronised-or-not) state,
    DS GPU vs the FP64 oracle on the same predicted positions."""
    import oracle
    from synth import sample_active
    st = ctx.nb_get_state()
    t_now = int(st["t"].max())
    n = m.shape[0]
    # predict everything to the latest particle time (FP64, the predictor of Section 2)
    dt = (t_now - st["t"]) / float(1 << 40)
    h = dt / 2.0
    q = dt / 3.0
    xp = st["x"] + (st["v"] + h[:, None] * (st["a"] + q[:, None] * st["k"])) * dt[:, None]
    vp = st["v"] + (st["a"] + h[:, None] * st["k"]) * dt[:, None]
    idx = sample_active(n, k, seed)
    ctx.nb_predict(t_now / float(1 << 40))
    got = ctx.nb_force(idx)
    ref = oracle.force(m, xp, vp, eps, idx, nthreads=os.cpu_count() or 1)
    sa, sk = pair_magnitude_sums(m, xp, vp, eps, idx)
    return force_error_stats(got, ref, sa, sk)


def run_adjoint(args):
    """Differentiable run: Plummer N = 16384 (seed 4), eps = 1/256, 256 shared
    Hermite steps of 1/1024, checkpoints every 16 steps, DS forward; loss =
    sum |x_T - x_target|^2 against a seeded Plummer snapshot (seed 5).
    Reports forward/backward times, gradients checked against FP64 central
    differences (h = 1e-6, GPU FP64 trajectory) on random coordinates, against
    the GPU FP64 adjoint, and against the CPU FP64 oracle adjoint at a size the
    sequential oracle finishes (stated)."""
    import torch
    import paper_cs_0702135_gb300 as nb
    torch.cuda.set_device(0)
    out = adjoint_config(nb, torch, args.n if args.n != N_DEFAULT else 16384, args.fd_coords,
                         args.oracle_n)
    print(json.dumps(out), flush=True)


def adjoint_config(nb, torch, n, fd_coords, oracle_n):
    from synth import plummer
    eps, level, steps, ck = 1.0 / 256, 10, 256, 16
    m, x, v = plummer(n, 4)
    tgt = plummer(n, 5)[1]
    out = {"workload": "adjoint_plummer_N%d_eps1/256_dt1/1024_steps%d_ckpt%d" % (n, steps, ck),
           "N": n, "steps": steps, "checkpoint_every": ck}

    def run(prec, xx=x, vv=v, mm=m, backward=True):
        c = nb.Context(mm, xx, vv, eps, precision=prec, level_fixed=level, flags=nb.NB_INIT_NO_FORCE)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.nb_traj_forward(steps, ck)
            xt = c.nb_get_state()["x"]
            t1 = time.perf_counter()
            loss = float(np.sum((xt - tgt) ** 2))
            if not backward:
                return loss
            g = c.nb_traj_backward(2 * (xt - tgt))
            t2 = time.perf_counter()
            return loss, g, t1 - t0, t2 - t1
        finally:
            c.nb_free()

    run(nb.NB_DS)   # warm-up (module load, allocations)
    loss, (gx, gv, gm), tf, tb = run(nb.NB_DS)
    pairs_f = (steps + 1) * n * (n - 1)
    out["ds"] = {"loss": loss, "forward_s": tf, "backward_s": tb,
                 "forward_interactions_per_s": pairs_f / tf,
                 "backward_pair_evaluations_per_s": (steps * n * (n - 1) + pairs_f) / tb,
                 "backward_over_forward": tb / tf}
    loss64, (hx, hv, hm), tf64, tb64 = run(nb.NB_FP64)
    out["fp64_gpu"] = {"loss": loss64, "forward_s": tf64, "backward_s": tb64}
    out["ds_vs_fp64_adjoint_rel_err"] = {
        "x": float(np.linalg.norm(gx - hx) / np.linalg.norm(hx)),
        "v": float(np.linalg.norm(gv - hv) / np.linalg.norm(hv)),
        "m": float(np.linalg.norm(gm - hm) / np.linalg.norm(hm))}
    # FP64 central differences on random coordinates of x0, v0 and m
    r = np.random.default_rng(7)
    h = 1e-6
    rows = []
    t_fd = time.perf_counter()
    for q in range(fd_coords):
        kind = ("x", "v", "m")[q % 3]
        i = int(r.integers(n))
        c3 = int(r.integers(3))
        xx, vv, mm = x.copy(), v.copy(), m.copy()
        if kind == "x":
            xx[i, c3] += h; lp = run(nb.NB_FP64, xx, vv, mm, False); xx[i, c3] -= 2 * h
            lm = run(nb.NB_FP64, xx, vv, mm, False); an_ds, an64 = gx[i, c3], hx[i, c3]
        elif kind == "v":
            vv[i, c3] += h; lp = run(nb.NB_FP64, xx, vv, mm, False); vv[i, c3] -= 2 * h
            lm = run(nb.NB_FP64, xx, vv, mm, False); an_ds, an64 = gv[i, c3], hv[i, c3]
        else:
            mm[i] += h; lp = run(nb.NB_FP64, xx, vv, mm, False); mm[i] -= 2 * h
            lm = run(nb.NB_FP64, xx, vv, mm, False); an_ds, an64 = gm[i], hm[i]
        fd = (lp - lm) / (2 * h)
        rows.append((kind, fd, an_ds, an64))
    t_fd = time.perf_counter() - t_fd
    scale = max([abs(r_[1]) for r_ in rows] + [1e-300])
    out["fd_check"] = {} if not rows else {"coords": len(rows), "h": h, "seconds": t_fd,
                       "max_abs_err_ds_over_max_fd": max(abs(r_[2] - r_[1]) for r_ in rows) / scale,
                       "max_abs_err_fp64_over_max_fd": max(abs(r_[3] - r_[1]) for r_ in rows) / scale,
                       "median_rel_err_ds": float(np.median([abs(r_[2] - r_[1]) / max(abs(r_[1]), 1e-30) for r_ in rows])),
                       "median_rel_err_fp64": float(np.median([abs(r_[3] - r_[1]) / max(abs(r_[1]), 1e-30) for r_ in rows]))}
    # CPU FP64 oracle adjoint at a smaller N (the oracle's pair loops are sequential)
    if oracle_n <= 0:
        return out
    import oracle
    no = oracle_n
    mo, xo, vo = plummer(no, 4)
    to = plummer(no, 5)[1]
    t0 = time.perf_counter()
    xt_o, _ = oracle.traj_final(mo, xo, vo, eps, 2.0 ** -level, steps)
    _, _, oxb, ovb, omb = oracle.traj_vjp(mo, xo, vo, eps, 2.0 ** -level, steps, 2 * (xt_o - to),
                                          np.zeros((no, 3)))
    t_orc = time.perf_counter() - t0
    c = nb.Context(mo, xo, vo, eps, level_fixed=level, flags=nb.NB_INIT_NO_FORCE)
    c.nb_traj_forward(steps, ck)
    xt_g = c.nb_get_state()["x"]
    gxo, gvo, gmo = c.nb_traj_backward(2 * (xt_g - to))
    c.nb_free()
    out["oracle_comparison"] = {"N": no, "oracle_seconds": t_orc,
                                "ds_rel_err_x": float(np.linalg.norm(gxo - oxb) / np.linalg.norm(oxb)),
                                "ds_rel_err_v": float(np.linalg.norm(gvo - ovb) / np.linalg.norm(ovb)),
                                "ds_rel_err_m": float(np.linalg.norm(gmo - omb) / np.linalg.norm(omb))}
    return out


def run_ensemble(args):
    """Batched ensemble: independent Plummer clusters (N log-uniform in
    [32, 4096], Salpeter masses on [0.1, 100], virial ratio uniform in
    [0.3, 0.7], seed 5), eps = 1/256, eta = 0.01, each to t = 1 with its own
    block steps; one graph-replayed launch per ensemble step, launch
    configuration from the autotuner.  Compared with per-cluster launches: the
    single-system path (nb_run per cluster), timed on a seeded sample of
    clusters and scaled to all of them."""
    import torch
    import paper_cs_0702135_gb300 as nb
    torch.cuda.set_device(0)
    fixed = tuple(int(q) for q in args.ens_config.split(",")) if args.ens_config else None
    print(json.dumps(ensemble_config(nb, torch, args.clusters, args.baseline_sample,
                                     oracle_outliers=args.oracle_outliers, fixed=fixed)), flush=True)


def ensemble_config(nb, torch, C, baseline_sample, oracle_outliers=0, oracle_n_max=512, fixed=None):
    from synth import ensemble
    t0 = time.perf_counter()
    cl = ensemble(C, 5, workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    off = np.zeros(C + 1, dtype=np.int64)
    for c, (m, _, _) in enumerate(cl):
        off[c + 1] = off[c] + m.shape[0]
    m = np.concatenate([c[0] for c in cl])
    x = np.concatenate([c[1] for c in cl])
    v = np.concatenate([c[2] for c in cl])
    eps = 1.0 / 256
    e = nb.Ensemble(off, m, x, v, eps)
    if fixed:
        th, gm = fixed
        e.nb_ens_configure(th, gm)
        ms_tuned = None
    else:
        th, gm, ms_tuned = e.nb_ens_tune(10)
    k0, p0 = e.nb_ens_energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    launches, inter = e.nb_ens_run(1.0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    k1, p1 = e.nb_ens_energy()
    st = e.nb_ens_get_state()
    e.nb_ens_free()
    dE = np.abs((k1 + p1) - (k0 + p0)) / np.abs(k0 + p0)
    sizes = np.diff(off)
    out = {"workload": "ensemble_%d_plummer_salpeter_N32-4096_eps1/256_t1" % C, "clusters": C,
           "particles": int(off[-1]), "generation_s": gen_s,
           "tuned": {"threads": th, "gmax": gm, "ms_per_step_at_start": ms_tuned},
           "launches": launches, "seconds": el, "clusters_per_s": C / el,
           "interactions": inter, "interactions_per_s": inter / el, "gflops": 60 * inter / el / 1e9,
           "steps_per_cluster": {"min": int(st["steps"].min()), "median": float(np.median(st["steps"])),
                                 "max": int(st["steps"].max())},
           "energy_rel_err": {"median": float(np.median(dE)), "p90": float(np.percentile(dE, 90)),
                              "max": float(dE.max()), "frac_le_1e-6": float(np.mean(dE <= 1e-6))},
           "all_at_t_end": bool(np.all(st["t"] == (1 << 40)))}
    if oracle_outliers > 0:
        out["oracle_outliers"] = ensemble_outliers_vs_oracle(cl, dE, eps, oracle_outliers, oracle_n_max)
    # per-cluster launches: the single-system path, one cluster at a time
    if baseline_sample <= 0:
        return out
    r = np.random.default_rng(55)
    pick = np.sort(r.choice(C, size=min(baseline_sample, C), replace=False))
    tb, ib = 0.0, 0
    for c in pick:
        mc, xc, vc = cl[c]
        ctx = nb.Context(mc, xc, vc, eps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it = ctx.nb_run(1.0)
        torch.cuda.synchronize()
        tb += time.perf_counter() - t0
        ib += it
        ctx.nb_free()
    out["per_cluster_launches"] = {"sample": int(len(pick)), "sample_seconds": tb,
                                   "sample_interactions": ib,
                                   "extrapolated_seconds": tb * C / len(pick),
                                   "clusters_per_s": len(pick) / tb,
                                   "ensemble_speedup_clusters_per_s": (C / el) / (len(pick) / tb)}
    return out


def ensemble_outliers_vs_oracle(cl, dE, eps, k, n_max):
    """The k clusters of at most n_max bodies with the largest GPU |dE/E|,
    each integrated to t = 1 by the oracle's FP64 integrator on the host
    cores: the oracle's own |dE/E| beside the GPU's."""
    import oracle
    thr = os.cpu_count() or 1
    cand = [c for c in np.argsort(-dE) if cl[c][0].shape[0] <= n_max][:k]
    rows = []
    for c in cand:
        m, x, v = cl[c]
        t0 = time.perf_counter()
        it = oracle.Integrator(m, x, v, 1.0 / 256, nthreads=thr)
        e0 = it.energy()
        steps, _, _ = it.run(1.0)
        d_orc = abs(it.energy() - e0) / abs(e0)
        rows.append({"cluster": int(c), "N": int(m.shape[0]), "m_max": float(m.max()),
                     "gpu_rel_err": float(dE[c]), "oracle_rel_err": d_orc, "oracle_steps": steps,
                     "oracle_seconds": time.perf_counter() - t0})
    return rows


# Wall-clock seconds for 0.25 N-body time units (t = 0.25 -> 0.5), equal-mass
# Plummer spheres, eps = 1/256, dt_max = 0.125: the paper's Tab:Results
# (GRAPE-6Af, GeForce 8800GTX through Cg/OpenGL, Quadro FX1400, one Xeon core).
PAPER_TAB_RESULTS = {
    256: (0.07098, 2.708, 3.423, 0.1325), 512: (0.1410, 8.777, 10.59, 0.5941),
    1024: (0.3327, 17.46, 20.20, 2.584), 2048: (0.7652, 45.27, 54.16, 10.59),
    4096: (1.991, 128.3, 157.8, 50.40), 8192: (5.552, 342.7, 617.3, 224.7),
    16384: (16.32, 924.4, 3398, 994.0), 32768: (51.68, 1907, 13180, 4328),
    65536: (178.2, 3973, 40560, 19290), 131072: (None, 8844, None, None),
    262144: (None, 22330, None, None), 524288: (None, 63960, None, None)}


def run_replay(args):
    """The paper's timing experiment (Section 4, Tab:Results) on this GPU: for
    each N, an equal-mass Plummer sphere (seed 7), eps = 1/256, dt_max = 0.125,
    eta = 0.01, integrated from t = 0 to 0.5 with block steps; the wall clock is
    measured over the last quarter, t = 0.25 -> 0.5, as in the paper."""
    import torch
    import paper_cs_0702135_gb300 as nb
    from synth import plummer
    torch.cuda.set_device(0)
    rows = []
    n = 256
    while n <= args.n_max:
        m, x, v = plummer(n, 7)
        ctx = nb.Context(m, x, v, 1.0 / 256)
        e0 = sum(ctx.nb_energy())
        ctx.nb_run(0.25)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, inter = ctx.nb_run(0.5)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e1 = sum(ctx.nb_energy())
        ctx.nb_free()
        paper = PAPER_TAB_RESULTS.get(n, (None,) * 4)
        rows.append({"N": n, "seconds_0.25_to_0.5": el, "steps": steps, "interactions": inter,
                     "interactions_per_s": inter / el, "mean_block": inter / max(1, steps) / (n - 1),
                     "energy_rel_err_0_to_0.5": abs(e1 - e0) / abs(e0),
                     "paper_seconds": {"grape6af": paper[0], "8800gtx": paper[1], "fx1400": paper[2],
                                       "xeon": paper[3]},
                     "speedup_vs_8800gtx": (paper[1] / el) if paper[1] else None})
        n *= 2
    print(json.dumps({"workload": "paper_tab_results_replay", "eps": 1.0 / 256, "rows": rows}), flush=True)


SUMMATIONS = (("compensated", 0), ("fixed", 1), ("fp32", 2), ("fp32_sorted", 3))
ACCURACY_SAMPLE = 256


def _rel_err_stats(got, ref):
    out = {}
    for name, g, r in zip(("acc", "jerk", "pot"), got, ref):
        g, r = np.asarray(g).reshape(len(r), -1), np.asarray(r).reshape(len(r), -1)
        e = np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)
        out[name] = {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)),
                     "max": float(e.max())}
    return out


def run_summation(args):
    """Summation variants (Section 6).  The timed step is the full-active block
    step of the default workload with GRAPE-style 64-bit fixed-point sums of
    the single-precision pair terms; beside it, every variant's force time and
    accuracy against the FP64 oracle on sampled particles, and the property
    that fixed point buys: bit-identical forces under a permutation of the
    particles and another j slicing."""
    import torch
    import oracle
    import paper_cs_0702135_gb300 as nb
    from synth import plummer, sample_active

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    n = args.n
    inter_per_step = n * (n - 1)

    m, x, v = plummer(n, SEED + rank)
    ctx = nb.Context(m, x, v, EPS, level_fixed=LEVEL, stream=stream.cuda_stream,
                     summation=nb.NB_SUM_FIXED)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    e0 = sum(ctx.nb_energy())
    for _ in range(args.warmup):
        flush.zero_()
        ctx.nb_step(wait=False)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(nvsmi_index(local))
    ctx.nb_get_stats(reset=True)
    ctx.nb_set_profiling(True)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        ctx.nb_step(wait=False)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    stats = ctx.nb_get_stats(reset=True)
    ctx.nb_set_profiling(False)
    if world > 1:
        elapsed = max_over_ranks(elapsed, dev)
        torch.distributed.barrier()
    e1 = sum(ctx.nb_energy())
    value = whole_job_rate(world, args.steps, inter_per_step, elapsed)

    force_s = stats["force_ms"] / 1e3 / max(1, stats["force_launches"])
    peak = fp32_peak_tflops(sms, MAX_SM_MHZ_FALLBACK)
    achieved = FLOP_PER_INTERACTION * inter_per_step / force_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": force_traffic_per_launch(n, "k_force_fixed.md", FIXED_SOURCES),
                "kernel": "k_force_fixed (full-N launch inside the step, with the bounds "
                          "reduction and combine around it)",
                "peak_note": "FP32 FMA peak 2 x 128 lanes x %d SMs x 2070 MHz (max SM clock); "
                             "achieved counts 60 flop per interaction although the variant issues "
                             "about 130 instructions per pair" % sms}
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / fp32_peak_tflops(sms, clocks["sm_mhz"])

    extras = {}
    if not args.no_extras and rank == 0:
        # every variant: force time on its own sample, accuracy on a common one
        idx_acc = sample_active(n, min(ACCURACY_SAMPLE, n), SEED + 17)
        ref = oracle.force(m, x, v, EPS, idx_acc, nthreads=os.cpu_count() or 1)
        variants, fixed_acc = {}, None
        for name, mode in SUMMATIONS:
            c = nb.Context(m, x, v, EPS, flags=nb.NB_INIT_NO_FORCE, stream=stream.cuda_stream,
                           summation=mode)
            na = {0: n, 1: n, 2: min(n, 4096), 3: min(n, 256)}[mode]
            idx = torch.from_numpy(sample_active(n, na, SEED + na)).to(dev)
            acc = torch.empty((na, 3), dtype=torch.float64, device=dev)
            jerk, pot = torch.empty_like(acc), torch.empty(na, dtype=torch.float64, device=dev)
            c.nb_force_dev(idx, na, acc, jerk, pot)
            c.nb_get_stats(reset=True)
            c.nb_set_profiling(True)
            for _ in range(2):
                c.nb_force_dev(idx, na, acc, jerk, pot)
            st = c.nb_get_stats(reset=True)
            fs = st["force_ms"] / 1e3 / max(1, st["force_launches"])
            got = c.nb_force(idx_acc)
            if mode == 1:
                fixed_acc = got
            c.nb_free()
            variants[name] = {"force_ms": fs * 1e3, "n_active": na,
                              "interactions_per_s": na * (n - 1) / fs,
                              "rel_err_vs_fp64": _rel_err_stats(got, ref)}
        # fixed point: the same bits for a permuted system sliced another way
        perm = np.random.default_rng(SEED).permutation(n)
        inv = np.argsort(perm).astype(np.int32)
        c = nb.Context(m[perm], x[perm], v[perm], EPS, flags=nb.NB_INIT_NO_FORCE,
                       stream=stream.cuda_stream, summation=nb.NB_SUM_FIXED, split_j=7)
        got_p = c.nb_force(inv[idx_acc])
        c.nb_free()
        same = all(np.array_equal(a, b) for a, b in zip(got_p, fixed_acc))
        extras["summation_variants"] = variants
        extras["fixed_bit_identical_under_permutation_and_split"] = bool(same)
        extras["accuracy_sample"] = "%d i drawn uniformly (seed %d) against all %d j, vs the FP64 oracle" % (
            len(idx_acc), SEED + 17, n)
        extras["e2e"] = e2e_host_api(ctx, nb, n, max(2, min(args.steps, 3)), torch, dev)
        if world == 1:
            rate, threads, na_s, secs = cpu_oracle_rate(m, x, v, EPS, summation=oracle.SUM_FIXED)
            extras["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                      "sample": "oracle fixed-point summation variant (OpenMP) on %d "
                                                "of the %d active i against all j, %.1f s" % (na_s, n, secs)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plummer_N%d_eps1/1024_full_active_block_step_fixed_point_sums" % n,
                   "N": n, "eps": EPS, "seed": SEED, "n_active": n, "shared_level": LEVEL,
                   "summation": "NB_SUM_FIXED: IEEE single-precision pair terms on double-single "
                                "positions, 64-bit fixed-point rounding, exact 128-bit sums",
                   "l2": "inputs larger than L2 and a 256 MiB memset between steps inside the "
                         "timed region",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "gflops": value * FLOP_PER_INTERACTION / 1e9,
        "pct_fp32_peak": 100.0 * value * FLOP_PER_INTERACTION / 1e12 / peak,
        "energy": {"rel_err": abs(e1 - e0) / abs(e0), "steps": args.warmup + args.steps,
                   "dt": 2.0 ** -LEVEL},
        "roofline": roofline,
        "gpu_launches": stats["kernel_launches"],
        "clocks": clocks,
        "device": {"name": props.name, "sms": sms},
    }
    line.update(extras)
    ctx.nb_free()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sweep(args):
    """Isolated force sweeps (the block sizes of a block-step run): for each
    n_active of --n-active, that many i against all N j of the default Plummer
    system.  value = the first block size's interactions/s; its roofline is the
    j-record stream (HBM) when the block is at most a few particles, else the
    FP32 ALU."""
    import torch
    import paper_cs_0702135_gb300 as nb
    from synth import plummer, sample_active

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    n = args.n
    nas = [int(a) for a in args.n_active.split(",")]
    if any(na < 1 or na > n for na in nas):
        raise SystemExit("--n-active entries must lie in [1, N]")
    m, x, v = plummer(n, SEED + rank)
    ctx = nb.Context(m, x, v, EPS, flags=nb.NB_INIT_NO_FORCE, stream=stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(nvsmi_index(local))
    sampler.start()
    ladder = time_sweeps(ctx, n, nas, dev, torch, sample_active, flush)
    clocks = sampler.stop()
    launches = sum(e["kernel_launches"] for e in ladder.values())
    first = ladder[str(nas[0])]
    if nas[0] <= SWEEP_HBM_MAX_ACTIVE:
        roofline = {"bound": "hbm", "achieved": first["j_record_gbs"], "peak": hbm_peak_gbs(),
                    "unit": "GB/s", "frac": first["j_record_hbm_frac"], "traffic": None,
                    "kernel": "k_force_jpar_ds (%d active i; algorithmic bytes: the 48-byte j "
                              "records of all N, read once)" % nas[0]}
    else:
        peak = fp32_peak_tflops(sms, MAX_SM_MHZ_FALLBACK)
        ach = FLOP_PER_INTERACTION * first["interactions_per_s"] / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None,
                    "kernel": "force kernels of a %d-particle block (60 flop per interaction)" % nas[0]}
    line = {
        "metric": "isolated force sweep: acc+jerk interactions/s", "value": first["interactions_per_s"],
        "unit": UNIT, "n_gpus": 1, "steps": sum(e["repetitions"] for e in ladder.values()),
        "warmup": 5 * len(nas), "ms_per_step": first["force_us"] / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plummer_N%d_eps1/1024_isolated_sweeps" % n, "N": n, "eps": EPS,
                   "seed": SEED, "n_active": nas,
                   "l2": "a 256 MiB memset before each repetition, outside the timed region"},
        "sweeps": ladder, "roofline": roofline, "gpu_launches": launches, "clocks": clocks,
        "device": {"name": props.name, "sms": sms},
    }
    ctx.nb_free()
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "blockstep":
        run_blockstep(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "replay":
        run_replay(args)
    elif args.workload == "summation":
        run_summation(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
