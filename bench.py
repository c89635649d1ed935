"""Benchmark: selected inversion of the 80^3 7-point grid Laplacian (n =
512,000, FP64) on one GB300, level-scheduled vs one supernode per launch.

One step = one full selected inversion (normalisation pass + every level
of the top-down sweep, Algorithm 3) of the already factored matrix, inputs
resident in HBM.  Factorisation and symbolic analysis happen once, before
the timed region (the paper times the phases separately, Section 4.2).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain column selected inversion) on a bounded sample of the same
workload family instead.  Multi-GPU (torchrun) runs independent replicas:
the method has no exchange step on one matrix in this design.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "selinv ms & FP64 TFLOP/s (frac of peak), batched vs plain, err<=1e-10"
# FP64 peak of this machine's GB300 when the live measurement below is not
# available: cuBLAS DGEMM 8192^3 (torch.matmul float64) measured at 1.10
# TFLOP/s, the same rate as mma.sync m8n8k4 f64 and DFMA.
FP64_PEAK_FALLBACK_TFLOPS = 1.10
# DRAM bytes of step 2 (all k_gemm1 launches of one sweep) over its
# algorithmic bytes, from a one-pass ncu capture of the 40^3 member of the
# family (profiles/k_gemm1_traffic_grid3d_40.md); the 80^3 traffic per launch
# is this ratio times the algorithmic bytes per launch.  Set to None whenever
# k_gemm1 changes until it is captured again.
STEP2_TRAFFIC_RATIO = 1.112


def measure_fp64_peak(dev, n=8192, reps=3):
    """cuBLAS DGEMM n^3 (torch.matmul float64) on this GPU: best of `reps`
    after one warm-up, TFLOP/s (the FP64 roofline denominator of this run)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def hbm_peak():
    """Measured copy bandwidth of this machine's GB300 (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def bf16_sustained_peak():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return float(json.load(f)["bf16_tflops_sustained"])


def emulated_step2_roofline(flops_gemm1, s2_ms):
    """Step-2 class of the opt-in emulated path (B' split, slice products,
    slice reductions) against the bf16 tensor peak: 28 bf16 slice products
    per multiply-add of X_{C,C} Lhat."""
    bf16 = 28 * flops_gemm1 / (s2_ms * 1e-3) / 1e12
    peak = bf16_sustained_peak()
    return {"bound": "tensor", "kernel": "step 2 emulated: k_em_split_lhat + k_em_gemm1 (mma.sync m16n8k16 "
                                         "bf16) + slice reductions",
            "achieved": bf16, "peak": peak, "unit": "TFLOP/s", "frac": bf16 / peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained", "traffic": None}


def factor_flops(sym):
    """Algorithmic flops of the supernodal LDL^T: per supernode (width s,
    |C| = r) r(r+1)s for the lower triangle of the Schur update
    L_CK D_K L_CK^T, r s^2 for the panel solve, 2/3 s^3 for the diagonal
    block (its LDL^T and the inverse of L_KK)."""
    s = np.diff(sym["sn_start"]).astype(float)
    r = np.diff(sym["rowptr"]).astype(float)
    return float(np.sum(r * (r + 1) * s + r * s * s + 2.0 / 3.0 * s ** 3))


def stats(xs):
    xs = list(xs)
    return {"median": statistics.median(xs), "std": statistics.pstdev(xs) if len(xs) > 1 else 0.0,
            "min": min(xs), "max": max(xs), "n": len(xs)}


WORKLOAD = ("grid3d_80: 80^3 7-point Laplacian, n=512000, diag 6+U(0.01,0.1), geometric nested "
            "dissection, relaxed supernodes of width <= 128, FP64")
# Oracle sample for the CPU baseline: the same grid family at a size the
# scalar oracle finishes in about 10 s on one core.
CPU_SAMPLE_SIDE = 32
CPU_WORKLOAD = ("grid3d_32 (CPU oracle sample of the grid3d_80 family): 32^3 7-point Laplacian, n=32768, "
                "diag 6+U(0.01,0.1), geometric nested dissection, relaxed supernodes of width <= 128, FP64")


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10, help="timed steps (one CUDA event pair each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=80)
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--class-steps", type=int, default=3,
                    help="steps of the separate pass with per-kernel-class events (roofline of step 2)")
    ap.add_argument("--factor-steps", type=int, default=3, help="timed factorisations (median)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end iterations (median)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="grid3d_80",
                    choices=["grid3d_80", "grid2d_31", "graphlap48", "dg_poles", "uneven48", "convdiff80",
                             "indefinite80"],
                    help="grid3d_80 is the headline; the others measure the remaining workload families")
    ap.add_argument("--poles", type=int, default=16, help="dg_poles: number of poles in the batch")
    ap.add_argument("--split-k-rows", type=int, default=None, help="override the library default")
    ap.add_argument("--small-cutoff", type=int, default=None, help="override the library default")
    ap.add_argument("--level-tiles", type=int, default=None, help="override the library default")
    ap.add_argument("--min-slice-rows", type=int, default=None, help="override the library default")
    ap.add_argument("--fp64-emulation", action="store_true",
                    help="experiments only: headline on the opt-in path with steps 2 and 3 emulated on the "
                         "bf16 tensor cores (opts.fp64_emulation = 1) instead of FP64 arithmetic")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device=None):
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, world, ms_max):
    """Throughput of N independent replicas timed by the slowest rank."""
    return flops_per_rank * world / (ms_max * 1e-3) / 1e12


def oracle_sample(side=CPU_SAMPLE_SIDE):
    """The oracle's factorisation of the side^3 member of the workload family
    (untimed) and the algorithmic flop count of its selected inversion."""
    import oracle
    import synth
    p = synth.grid3d(side)
    sym = oracle.analyse(p.n, p.colptr, p.rowind, 128, 1)
    lcp, lri = oracle.supernodal_pattern(p.n, sym["sn_start"], sym["rcount"], sym["rrows"])
    lv, d = oracle.ldlt(p.n, sym["colptr"], sym["rowind"], p.values, lcp, lri)
    s = np.diff(sym["sn_start"]).astype(float)
    r = sym["rcount"].astype(float)
    flops = float(np.sum(2 * r * r * s + 3 * r * s * s + 2.0 / 3.0 * s ** 3))
    return p.n, lcp, lri, lv, d, flops


def time_oracle_selinv(sample, threads=None):
    """Seconds of one oracle column selected inversion of the sample
    (threads=None: the plain single-thread recurrence; else its OpenMP
    row/column-parallel variant on that many threads, bitwise the same X)."""
    import oracle
    n, lcp, lri, lv, d, _ = sample
    t0 = time.perf_counter()
    oracle.selinv(n, lcp, lri, lv, d, threads=threads)
    return time.perf_counter() - t0


def cpu_baseline_block():
    """The oracle on this host's cores: one run on 1 thread and one
    on all cores (nproc) of the 32^3 sample (~10 s of CPU work in total)."""
    sample = oracle_sample()
    flops = sample[-1]
    cores = host_cores()
    t1 = time_oracle_selinv(sample)
    tn = time_oracle_selinv(sample, threads=cores)
    return {"value": flops / tn / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "seconds": tn, "value_1_thread": flops / t1 / 1e12, "seconds_1_thread": t1,
            "sample": f"oracle column selected inversion (factorisation untimed) of the {CPU_SAMPLE_SIDE}^3 member "
                      f"of the same grid family ({flops:.3e} algorithmic flops), on {cores} threads (OpenMP, "
                      f"bitwise the single-thread result) and on 1 thread"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    sample = oracle_sample()
    flops = sample[-1]
    cores = host_cores()
    for _ in range(args.warmup):
        time_oracle_selinv(sample, threads=cores)
    secs = [time_oracle_selinv(sample, threads=cores) for _ in range(args.steps)]
    ms = 1e3 * sum(secs) / len(secs)
    value = flops / (ms * 1e-3) / 1e12
    desc = (f"oracle column selected inversion on {cores} host threads (OpenMP; factorisation untimed) of the "
            f"{CPU_SAMPLE_SIDE}^3 grid, n={CPU_SAMPLE_SIDE ** 3}; TFLOP/s by the supernodal algorithmic flop "
            f"count of that instance ({flops:.3e})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_stats": stats(1e3 * x for x in secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": CPU_WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].isdigit():
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace('.', '').isdigit())
                if any(r[3].replace('.', '').isdigit() for r in rows) else None}


def tuning(args):
    kw = {}
    if args.split_k_rows is not None:
        kw["split_k_rows"] = args.split_k_rows
    if args.small_cutoff is not None:
        kw["small_cutoff"] = args.small_cutoff
    if args.level_tiles is not None:
        kw["level_tiles"] = args.level_tiles
    if args.min_slice_rows is not None:
        kw["min_slice_rows"] = args.min_slice_rows
    if args.fp64_emulation:
        kw["fp64_emulation"] = 1
    return kw


def run_ours(args):
    import torch
    import torch.distributed as dist
    import synth
    import paper_1404_0447_gb300 as P

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load_library()

    prob = synth.grid3d(args.side)
    h = P.SelInv(prob.n, prob.colptr, prob.rowind, max_sn_width=128, relax=P.RELAX_AMALG, **tuning(args))
    info = h.info
    sym = h.symbolic()
    flops = info["flops_selinv"]
    vals = torch.tensor(prob.values, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    h.factor(vals, stream=stream)
    h.sync_status(stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(mode, steps):
        """K steps with one event pair per step and one around all of them,
        bracketed by a barrier and a device synchronisation on both sides:
        (ms per step over the whole region, per-step ms list)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            h.selinv(mode, stream=stream)
            ev[k][1].record(stream)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1) / steps, [a.elapsed_time(b) for a, b in ev]

    peak = None
    if not args.fp64_emulation:
        peak = measure_fp64_peak(dev)
    peak_used = peak if peak else FP64_PEAK_FALLBACK_TFLOPS

    # warm-up (level schedule)
    for _ in range(args.warmup):
        h.selinv(P.LEVEL, stream=stream)
    torch.cuda.synchronize()

    # headline: level-scheduled sweep, nothing else recorded in the timed region
    with ClockSampler(local) as clk:
        ms, per_step = timed(P.LEVEL, args.steps)
    clocks = clk.summary()
    ms = max_over_ranks(ms, dev)
    value = whole_job_tflops(flops, world, ms)

    # separate pass with per-kernel-class events (launch counts, step-2 roofline)
    csteps = max(1, args.class_steps)
    h.set_timing(True)
    ms_inst, _ = timed(P.LEVEL, csteps)
    kms, kl = h.get_timing()
    h.set_timing(False)
    kms, kl = kms / csteps, kl / csteps

    # graph-replayed level schedule, persistent schedule, plain one-supernode-per-launch schedule
    h.selinv(P.GRAPH, stream=stream)
    torch.cuda.synchronize()
    ms_graph, _ = timed(P.GRAPH, max(1, min(args.steps, 5)))
    ms_persistent = None
    if not args.fp64_emulation:  # the persistent kernel runs the FP64 steps only
        h.selinv(P.PERSISTENT, stream=stream)
        h.sync_status(stream=stream)
        ms_persistent, _ = timed(P.PERSISTENT, max(1, min(args.steps, 5)))
        h.sync_status(stream=stream)
    ms_plain = None
    if not args.no_plain:
        h.selinv(P.PLAIN, stream=stream)
        torch.cuda.synchronize()
        ms_plain, _ = timed(P.PLAIN, max(1, args.plain_steps))

    # the index-driven gather of the selected entries at A's positions (HBM-bound):
    # per entry the int64 value-map offset, the X panel value and the output
    sel_out = torch.empty(info["nnz_a"], dtype=torch.float64, device=dev)
    h.selected(out=sel_out, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        h.selected(out=sel_out, stream=stream)
    e1.record(stream)
    e1.synchronize()
    g_ms = e0.elapsed_time(e1) / 10
    gather_block = {"kernel": "k_gather_values (selected entries of X at A's nonzeros)", "ms": g_ms,
                    "bytes": 24 * info["nnz_a"], "achieved_GBps": 24 * info["nnz_a"] / (g_ms * 1e-3) / 1e9,
                    "peak_GBps": hbm_peak(), "frac": 24 * info["nnz_a"] / (g_ms * 1e-3) / 1e9 / hbm_peak()}
    del sel_out

    # the factorisation on resident values (the step before the path; timed separately)
    fl_factor = factor_flops(sym)
    fms = []
    for _ in range(max(1, args.factor_steps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.factor(vals, stream=stream)
        e1.record(stream)
        e1.synchronize()
        fms.append(e0.elapsed_time(e1))
    h.sync_status(stream=stream)
    f_med = statistics.median(fms)
    factor_block = {"bound": "tensor", "kernel": "pselinv_factor: k_factor_diag, k_trsm, k_copyback, k_schur "
                                                "(FP64 mma.sync m8n8k4) per level, Schur updates in groups "
                                                "with disjoint targets (no atomics)",
                    "flops": fl_factor, "ms_stats": stats(fms), "achieved": fl_factor / (f_med * 1e-3) / 1e12,
                    "peak": peak_used, "unit": "TFLOP/s", "frac": fl_factor / (f_med * 1e-3) / 1e12 / peak_used,
                    "flop_count": "sum over supernodes of r(r+1)s + r s^2 + 2/3 s^3"}

    # end to end through host buffers: values H2D, factor, selinv, X panels D2H
    e2e = None
    if not args.no_e2e:
        host_vals = torch.tensor(prob.values, dtype=torch.float64).pin_memory()
        host_out = torch.empty(info["panel_entries"], dtype=torch.float64).pin_memory()
        dev_vals = torch.empty_like(vals)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        walls, ph = [], []
        for it in range(max(1, args.e2e_steps)):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                dev_vals.copy_(host_vals, non_blocking=True)
                ev[1].record(stream)
                h.factor(dev_vals, stream=stream)
                ev[2].record(stream)
                # LEVEL selinv; each finished level's X panels go to pinned host memory meanwhile
                h.selinv_to_host(host_out, stream=stream)
                ev[3].record(stream)
            stream.synchronize()
            walls.append(1e3 * (time.perf_counter() - t0))
            ph.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
        h.sync_status(stream=stream)
        t_med = statistics.median(walls)
        phases = {name: statistics.median(p[i] for p in ph)
                  for i, name in enumerate(("h2d_ms", "factor_ms", "selinv_and_d2h_ms"))}
        phases["d2h_exposed_ms"] = phases["selinv_and_d2h_ms"] - ms
        e2e = {"value": whole_job_tflops(flops, world, max_over_ranks(t_med, dev)), "unit": "TFLOP/s",
               "ms_per_step": t_med, "ms_stats": stats(walls),
               "h2d_bytes_per_step": int(host_vals.numel() * 8), "d2h_bytes_per_step": int(host_out.numel() * 8),
               "includes": "pinned H2D of A's values, pselinv_factor, pselinv_selinv_to_host (LEVEL selinv with "
                           "the X panels of each finished level copied to pinned host memory during the sweep); "
                           "wall clock per iteration, median",
               "phases": phases}

    # roofline of the dominant kernel (step 2, X_{C,K} = -X_{C,C} Lhat): algorithmic
    # flops per launch over its event-timed average launch duration (separate pass)
    g1_launches = max(1, int(round(kl[1])))
    g1_ms_launch = kms[1] / g1_launches
    achieved = info["flops_gemm1"] / g1_launches / (g1_ms_launch * 1e-3) / 1e12
    sw = np.diff(sym["sn_start"]).astype(float)
    rr = np.diff(sym["rowptr"]).astype(float)
    rel = np.diff(sym["relptr"]).astype(float)
    g1_alg_bytes = float(np.sum(8 * rr * (rr + 1) / 2 + 16 * rr * sw + 4 * rel))
    default_schedule = (args.split_k_rows is None and args.small_cutoff is None and args.level_tiles is None
                        and args.min_slice_rows is None and args.side == 80)
    roofline = {"bound": "tensor",
                "kernel": "step 2: k_gemm1 (all tile widths, FP64 mma.sync m8n8k4, which runs on the FP64 pipe "
                          "of sm_103a) + slice reductions",
                "achieved": achieved, "peak": peak_used, "unit": "TFLOP/s", "frac": achieved / peak_used,
                "peak_source": ("cuBLAS DGEMM 8192^3 (torch.matmul float64) measured in this run, best of 3 (FP64 "
                                "has no entry in MEASURED_PEAKS.json)") if peak else
                               "fallback 1.10 TFLOP/s: cuBLAS DGEMM measured earlier on this pool",
                "traffic": (STEP2_TRAFFIC_RATIO * g1_alg_bytes / g1_launches
                            if default_schedule and STEP2_TRAFFIC_RATIO else None),
                "traffic_unit": "DRAM bytes per launch: DRAM/algorithmic ratio of a one-pass ncu capture of the "
                                "40^3 member (%s) times the algorithmic bytes per launch" % STEP2_TRAFFIC_RATIO,
                "algorithmic_bytes_per_launch": g1_alg_bytes / g1_launches,
                "launches_per_step": g1_launches,
                "timing": "per-kernel-class CUDA events on the launching stream, in a separate pass of %d steps "
                          "(%.1f ms per step with the events, %.1f ms without)" % (csteps, ms_inst, ms),
                "whole_step_frac": value / world / peak_used}
    if args.fp64_emulation:
        roofline = dict(emulated_step2_roofline(info["flops_gemm1"], kms[1]),
                        whole_step_fp64_equivalent_tflops=value / world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64" if not args.fp64_emulation else "f64 (steps 2, 3: bf16 slice products, exact integer sums)",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": prob.n, "nnz_a_lower": info["nnz_a"],
                           "nnz_l": info["nnz_l"], "supernodes": info["nsn"], "levels": info["nlevels"],
                           "flops_per_step": flops, "schedule": "level (one grouped launch per kernel per level)",
                           "ms_stats": stats(per_step),
                           "batched_ms": ms, "graph_ms": ms_graph, "persistent_ms": ms_persistent, "plain_ms": ms_plain,
                           "speedup_batched_vs_plain": ms_plain / ms if ms_plain else None,
                           "kernel_ms_per_step": {"normalise": kms[0], "step2_gemm1": kms[1],
                                                  "step3_partials": kms[2], "step3_finish": kms[3]},
                           "fp64_peak_measured_tflops": peak,
                           "l2": "no flush: the X panels (%.1f GB) exceed L2 (129 MB)" % (info["panel_entries"] * 8 / 1e9),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "factor": factor_block, "gather": gather_block, "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": int(round(sum(kl))) * args.steps, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _time(fn, steps, warmup, stream):
    """Device time per call of fn() on `stream`, after warm-up (CUDA events)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def run_workload(args):
    """Secondary workloads (one JSON line each): level / graph / plain selinv
    times, TFLOP/s (complex counted x4), and for graphlap48 the logdet
    forward, backward and adjoint times."""
    import torch
    import synth
    import paper_1404_0447_gb300 as P
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    P.load_library()
    w = args.workload
    peak = measure_fp64_peak(dev)
    line = {"workload": w, "steps": args.steps, "warmup": args.warmup, "fp64_peak_measured_tflops": peak}
    if w == "grid2d_31":
        p = synth.grid2d_31()
        h = P.SelInv(p.n, p.colptr, p.rowind, max_sn_width=128, relax=P.RELAX_NONE, **tuning(args))
        vals = torch.tensor(p.values, dtype=torch.float64, device=dev)
        cplx = False
    elif w == "graphlap48":
        gl = synth.GraphLaplacian((48, 48, 48))
        h = P.SelInv(gl.n, gl.colptr, gl.rowind, perm=synth.nd_order(gl.dims), **tuning(args))
        vals = torch.tensor(gl.assemble(), dtype=torch.float64, device=dev)
        cplx = False
    elif w == "dg_poles":
        n, cp, ri, hv, z = synth.dg_block_matrix((12, 12, 12), 48, 16)
        z = z[:args.poles]
        h = P.SelInv(n, cp, ri, perm=synth.block_nd_order((12, 12, 12), 48), dtype=P.C128, batch=len(z),
                     **tuning(args))
        vals = torch.tensor(synth.shifted_values(n, cp, ri, hv, z), dtype=torch.complex128, device=dev)
        cplx = True
        line["poles"] = len(z)
    elif w == "indefinite80":
        # symmetric indefinite: the 80^3 grid Laplacian shifted by -0.5 into its spectrum
        # (2,908 negative eigenvalues), factored with Bunch-Kaufman 1x1/2x2 pivots inside supernodes
        p = synth.grid3d(80, shift_const=-0.5)
        h = P.SelInv(p.n, p.colptr, p.rowind, **tuning(args))
        vals = torch.tensor(p.values, dtype=torch.float64, device=dev)
        cplx = False
    elif w == "convdiff80":
        # non-symmetric: 80^3 upwind convection-diffusion, A = L D U', Algorithm 1 with step 4
        p = synth.convdiff_problem(80)
        h = P.SelInv(p.n, p.colptr, p.rowind, unsym=1, **tuning(args))
        vals = torch.tensor(p.values, dtype=torch.float64, device=dev)
        vals_up = torch.tensor(p.values_up, dtype=torch.float64, device=dev)
        cplx = False
    else:
        mem = [synth.uneven_member(s) for s in synth.uneven_batch_specs()]
        h = P.SelInv([m.n for m in mem], [m.colptr for m in mem], [m.rowind for m in mem], **tuning(args))
        vals = torch.tensor(np.concatenate([m.values for m in mem]), dtype=torch.float64, device=dev)
        cplx = False
    info = h.info
    flops = info["flops_selinv"] * info["batch"] * (4 if cplx else 1)
    line.update({k: info[k] for k in ("n", "nnz_l", "nsn", "nlevels", "batch")})
    line["flops_per_selinv"] = flops
    unsym = w == "convdiff80"
    factor = ((lambda: h.factor_unsym(vals, vals_up, stream=st)) if unsym
              else (lambda: h.factor_bk(vals, stream=st)) if w == "indefinite80"
              else (lambda: h.factor(vals.view(-1), stream=st)))
    with torch.cuda.stream(st):
        factor()
        h.sync_status(stream=st)
        line["factor_ms"] = _time(factor, max(1, args.factor_steps), 0, st)
        h.sync_status(stream=st)
    # factor flops: r(r+1)s + r s^2 + 2/3 s^3 per supernode (non-symmetric: both sides,
    # 2 r^2 s + 2 r s^2 + 4/3 s^3), complex x4, times the batch
    fsym = h.symbolic()
    fs = np.diff(fsym["sn_start"]).astype(float)
    fr = np.diff(fsym["rowptr"]).astype(float)
    ff = (np.sum(2 * fr * fr * fs + 2 * fr * fs * fs + 4.0 / 3.0 * fs ** 3) if unsym
          else factor_flops(fsym)) * info["batch"] * (4 if cplx else 1)
    line["factor_tflops"] = ff / (line["factor_ms"] * 1e-3) / 1e12
    line["factor_frac_of_fp64_peak"] = line["factor_tflops"] / peak
    for name, mode in (("level", P.LEVEL), ("graph", P.GRAPH), ("persistent", P.PERSISTENT), ("plain", P.PLAIN)):
        if w == "dg_poles" and args.poles > 4 and name != "level":
            continue  # ~150 s per selinv at 16 poles: the level schedule only
        if unsym and mode == P.PERSISTENT:
            continue  # the persistent schedule is for symmetric handles
        if args.no_plain and mode == P.PLAIN:
            continue
        ms = _time(lambda: h.selinv(mode, stream=st), args.steps if name != "plain" else 1,
                   args.warmup if name != "plain" else 1, st)
        line[f"{name}_ms"] = ms
        line[f"{name}_tflops"] = flops / (ms * 1e-3) / 1e12
        line[f"{name}_frac_of_fp64_peak"] = line[f"{name}_tflops"] / peak
    if "plain_ms" in line:
        line["speedup_level_vs_plain"] = line["plain_ms"] / line["level_ms"]
    if w == "dg_poles":
        # pole expansion Gamma = sum_l w_l X_l (weights 1/P here) and E(z_l) of Eq. (16)
        wts = np.full(info["batch"], 1.0 / info["batch"], np.complex128)
        gam = torch.empty(info["panel_entries"], dtype=torch.complex128, device=dev)
        line["pole_sum_ms"] = _time(lambda: h.pole_sum(wts, out=gam, stream=st), 3, 1, st)
        line["pole_sum_GBps"] = (info["batch"] + 1) * info["panel_entries"] * 16 / (line["pole_sum_ms"] * 1e-3) / 1e9
        # the same sum accumulated in the sweep's write step: selinv + Gamma in one call
        line["selinv_pole_sum_fused_ms"] = _time(lambda: h.selinv_pole_sum(wts, out=gam, stream=st), 1, 1, st)
        line["trace_E_per_pole"] = [float(e) for e in h.trace_error(vals.view(-1), stream=st)]
    if w == "indefinite80":
        piv, ty = h.pivots(stream=st)
        line["pivots_2x2"] = int((ty == 1).sum())
        line["pivots_interchanged"] = int(np.sum(piv[0] != (np.arange(p.n) - np.repeat(
            np.asarray(h.symbolic()["sn_start"][:-1]), np.diff(h.symbolic()["sn_start"])))))
    if not (w == "dg_poles" and args.poles > 4):
        # kernel classes of one level-schedule selinv (class 1 = step 2, and step 4 when non-symmetric)
        h.set_timing(True)
        h.selinv(P.LEVEL, stream=st)
        kms, kl = h.get_timing()
        h.set_timing(False)
        s2 = "step2_step4" if unsym else "step2"
        line["kernel_ms"] = {"normalise": kms[0], s2: kms[1], "step3_partials": kms[2], "step3_finish": kms[3]}
        line["kernel_launches"] = [int(x) for x in kl]
        line[f"{s2}_tflops"] = info["flops_gemm1"] * info["batch"] * (4 if cplx else 1) / (kms[1] * 1e-3) / 1e12
        line[f"{s2}_frac_of_fp64_peak"] = line[f"{s2}_tflops"] / peak
    if w == "graphlap48":
        # differentiable logdet: forward = factor + logdet, backward = selinv + gradient gather
        g = torch.empty(info["nnz_a"], dtype=torch.float64, device=dev)
        line["logdet_forward_ms"] = _time(lambda: (h.factor(vals, stream=st), h.logdet(stream=st)), 3, 1, st)
        line["logdet_backward_ms"] = _time(lambda: (h.selinv(P.LEVEL, stream=st), h.logdet_grad(out=g, stream=st)),
                                           args.steps, 1, st)
        G = torch.randn(info["panel_entries"], dtype=torch.float64, device=dev)
        h.selinv(P.LEVEL, stream=st)
        line["adjoint_ms"] = _time(lambda: h.adjoint(G, stream=st), 3, 1, st)
        # adjoint work per supernode: r^2 s terms -X_CC Yb, the scatter -(Yb Lhat^T + Lhat Yb^T)
        # (lower triangle) and (W + W^T) L_CK; r s^2 terms Ybar, Y Zb^T, Hb V^T, L_CK^T Hb, the
        # solve with V and Q^T L_CK; six s x s products of the diagonal steps
        asym = h.symbolic()
        a_s = np.diff(asym["sn_start"]).astype(float)
        a_r = np.diff(asym["rowptr"]).astype(float)
        adj_flops = float(np.sum(6 * a_r * a_r * a_s + 2 * a_r * a_s + 10 * a_r * a_s * a_s
                                 + 6 * a_s * a_s * (a_s + 1)))
        line["adjoint_flops"] = adj_flops
        line["adjoint_tflops"] = adj_flops / (line["adjoint_ms"] * 1e-3) / 1e12
        line["adjoint_frac_of_fp64_peak"] = line["adjoint_tflops"] / peak
    if w == "uneven48":
        # the same members one handle at a time (level schedule each)
        hs = []
        for m in mem:
            hm = P.SelInv(m.n, m.colptr, m.rowind)
            hm.factor(torch.tensor(m.values, dtype=torch.float64, device=dev), stream=st)
            hs.append(hm)
        torch.cuda.synchronize()
        ms = _time(lambda: [hm.selinv(P.LEVEL, stream=st) for hm in hs], 2, 1, st)
        line["per_member_level_ms"] = ms
        line["speedup_merged_graph_vs_per_member"] = ms / line["graph_ms"]
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "grid3d_80":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
