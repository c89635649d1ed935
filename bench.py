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
# FP64 peak measured on this machine's GB300: cuBLAS DGEMM 8192^3 (torch.matmul
# float64) and mma.sync m8n8k4 f64 throughput both ~1.10 TFLOP/s; see
# profiles/fp64_peak_gb300.md.
FP64_PEAK_TFLOPS = 1.10
# DRAM bytes per step-2 launch (all k_gemm1 widths and slice reductions) at
# the full 80^3 workload with the default schedule, from one-pass ncu
# counters: profiles/k_gemm1_traffic_grid3d_80.md.  Set to None whenever
# those kernels change until they are measured again.
STEP2_TRAFFIC_BYTES_PER_LAUNCH = 460.55e6
# bf16 dense peaks: MEASURED_PEAKS.json (cuBLAS, sustained over seconds) and
# the warp-level mma.sync m16n8k16 rate of the same GPU (bench.py --peaks).
MEASURED_BF16_SUSTAINED_TFLOPS = 1696.4
MMA_SYNC_BF16_TFLOPS = 605.7


def bf16_sustained_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError):
        return MEASURED_BF16_SUSTAINED_TFLOPS


def emulated_step2_roofline(flops_gemm1, s2_ms):
    """Step-2 class of the emulated path (B' split, slice products, slice
    reductions) against the bf16 tensor peak: 28 bf16 slice products per
    multiply-add of X_{C,C} Lhat."""
    bf16 = 28 * flops_gemm1 / (s2_ms * 1e-3) / 1e12
    peak = bf16_sustained_peak()
    return {"bound": "tensor", "kernel": "step 2 emulated: k_em_split_lhat + k_em_gemm1 (mma.sync m16n8k16 "
                                         "bf16) + slice reductions",
            "achieved": bf16, "peak": peak, "unit": "TFLOP/s", "frac": bf16 / peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS); the warp-level mma.sync path of "
                           "this GPU tops out near %.0f (bench.py --peaks)" % MMA_SYNC_BF16_TFLOPS,
            "frac_of_mma_sync_peak": bf16 / MMA_SYNC_BF16_TFLOPS, "traffic": None}
WORKLOAD = ("grid3d_80: 80^3 7-point Laplacian, n=512000, diag 6+U(0.01,0.1), geometric nested "
            "dissection, relaxed supernodes of width <= 128, FP64")
# Oracle sample for the CPU baseline: the same grid family at a size the
# scalar oracle finishes in about 10-30 s.
CPU_SAMPLE_SIDE = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=80)
    ap.add_argument("--plain-steps", type=int, default=1)
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
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 and low-precision MMA peaks of this GPU (the roofline denominators)")
    ap.add_argument("--min-slice-rows", type=int, default=None, help="override the library default")
    ap.add_argument("--fp64-emulation", action="store_true",
                    help="headline on the opt-in path with step 2 emulated on the bf16 tensor cores "
                         "(opts.fp64_emulation = 1) instead of FP64 arithmetic")
    ap.add_argument("--emulation-variant", type=int, default=1, choices=[1, 2],
                    help="emulated step 2 on mma.sync (1) or tcgen05 (2)")
    ap.add_argument("--no-emulation", action="store_true",
                    help="skip the secondary measurement of the emulated step 2 (config.fp64_emulation)")
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


def oracle_sample_tflops(side=CPU_SAMPLE_SIDE):
    """Time the oracle's column selected inversion (its factorisation done
    first, untimed) on the side^3 member of the workload family; return
    (TFLOP/s by the algorithmic count of that instance, seconds, flops)."""
    import oracle
    import synth
    p = synth.grid3d(side)
    sym = oracle.analyse(p.n, p.colptr, p.rowind, 128, 1)
    lcp, lri = oracle.supernodal_pattern(p.n, sym["sn_start"], sym["rcount"], sym["rrows"])
    lv, d = oracle.ldlt(p.n, sym["colptr"], sym["rowind"], p.values, lcp, lri)
    s = np.diff(sym["sn_start"]).astype(float)
    r = sym["rcount"].astype(float)
    flops = float(np.sum(2 * r * r * s + 3 * r * s * s + 2.0 / 3.0 * s ** 3))
    t0 = time.perf_counter()
    oracle.selinv(p.n, lcp, lri, lv, d)
    dt = time.perf_counter() - t0
    return flops / dt / 1e12, dt, flops


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    sample = (f"oracle column selected inversion (single thread, factorisation untimed) of the "
              f"{CPU_SAMPLE_SIDE}^3 member of the same 7-point grid family (n={CPU_SAMPLE_SIDE ** 3}); "
              f"TFLOP/s by the supernodal algorithmic flop count of that instance")
    for _ in range(args.warmup):
        oracle_sample_tflops()
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, fl = oracle_sample_tflops()
        vals.append(v)
        secs.append(dt)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
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
        kw["fp64_emulation"] = args.emulation_variant
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
    flops = info["flops_selinv"]
    vals = torch.tensor(prob.values, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        h.factor(vals, stream=stream)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(mode, steps, record=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        if record:
            h.set_timing(True)
        e0.record(stream)
        for _ in range(steps):
            h.selinv(mode, stream=stream)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        kt = h.get_timing() if record else None
        if record:
            h.set_timing(False)
        return ms, kt

    # warm-up (level schedule, also captures nothing)
    for _ in range(args.warmup):
        h.selinv(P.LEVEL, stream=stream)
    torch.cuda.synchronize()

    # headline: level-scheduled sweep, kernel classes bracketed by events
    with ClockSampler(local) as clk:
        ms, (kms, kl) = timed(P.LEVEL, args.steps, record=True)
    clocks = clk.summary()
    ms = max_over_ranks(ms, dev)

    # graph-replayed level schedule and the plain one-supernode-per-launch schedule
    h.selinv(P.GRAPH, stream=stream)
    torch.cuda.synchronize()
    ms_graph, _ = timed(P.GRAPH, max(1, args.steps))
    ms_persistent = None
    if not args.fp64_emulation:  # the persistent kernel runs the FP64 step 2 only
        h.selinv(P.PERSISTENT, stream=stream)
        h.sync_status(stream=stream)
        ms_persistent, _ = timed(P.PERSISTENT, max(1, args.steps))
    h.sync_status(stream=stream)
    ms_plain = None
    if not args.no_plain:
        h.selinv(P.PLAIN, stream=stream)
        torch.cuda.synchronize()
        ms_plain, _ = timed(P.PLAIN, max(1, args.plain_steps))

    # end to end through host buffers: values H2D, factor, selinv, X panels D2H
    e2e = None
    if not args.no_e2e:
        host_vals = torch.tensor(prob.values, dtype=torch.float64).pin_memory()
        host_out = torch.empty(info["panel_entries"], dtype=torch.float64).pin_memory()
        dev_vals = torch.empty_like(vals)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for it in range(3):
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
            t_e2e = time.perf_counter() - t0
        phases = {name: ev[i].elapsed_time(ev[i + 1])
                  for i, name in enumerate(("h2d_ms", "factor_ms", "selinv_and_d2h_ms"))}
        phases["d2h_exposed_ms"] = phases["selinv_and_d2h_ms"] - ms
        e2e = {"value": whole_job_tflops(flops, world, max_over_ranks(1e3 * t_e2e, dev)), "unit": "TFLOP/s",
               "ms_per_step": 1e3 * t_e2e,
               "h2d_bytes_per_step": int(host_vals.numel() * 8), "d2h_bytes_per_step": int(host_out.numel() * 8),
               "includes": "pinned H2D of A's values, pselinv_factor, pselinv_selinv_to_host (LEVEL selinv with "
                           "the X panels of each finished level copied to pinned host memory during the sweep)",
               "phases": phases}

    # secondary: the opt-in step 2 emulated on the bf16 tensor cores, on its own
    # handle, against this handle's FP64 X (not the headline: FP64 arithmetic is)
    emul = None
    if not args.fp64_emulation and not args.no_emulation:
        emul = measure_emulation(args, prob, info, vals, h, stream, dev)

    value = whole_job_tflops(flops, world, ms)
    # roofline of the dominant kernel (step 2, X_{C,K} = -X_{C,C} Lhat): algorithmic
    # flops per launch over its event-timed average launch duration
    g1_launches = max(1, int(kl[1]) // args.steps)
    g1_ms_launch = kms[1] / args.steps / g1_launches
    g1_flops_launch = info["flops_gemm1"] / g1_launches
    achieved = g1_flops_launch / (g1_ms_launch * 1e-3) / 1e12
    sym = h.symbolic()
    sw = np.diff(sym["sn_start"]).astype(float)
    rr = np.diff(sym["rowptr"]).astype(float)
    rel = np.diff(sym["relptr"]).astype(float)
    g1_alg_bytes = float(np.sum(8 * rr * (rr + 1) / 2 + 16 * rr * sw + 4 * rel))
    default_schedule = (args.split_k_rows is None and args.small_cutoff is None and args.level_tiles is None
                        and args.min_slice_rows is None and args.side == 80)
    roofline = {"bound": "tensor",
                "kernel": "step 2: k_gemm1 (all tile widths, FP64 mma.sync m8n8k4, which runs on the FP64 pipe "
                          "of sm_103a) + slice reductions",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "measured cuBLAS DGEMM / mma.sync f64 throughput on this pool's GB300 (FP64 has no "
                               "entry in MEASURED_PEAKS.json)",
                "traffic": STEP2_TRAFFIC_BYTES_PER_LAUNCH if default_schedule else None,
                "traffic_unit": "DRAM bytes per launch (ncu, one pass, full workload)",
                "algorithmic_bytes_per_launch": g1_alg_bytes / g1_launches,
                "launches_per_step": g1_launches,
                "whole_step_frac": value / world / FP64_PEAK_TFLOPS}
    if args.fp64_emulation:
        roofline = dict(emulated_step2_roofline(info["flops_gemm1"], kms[1] / args.steps),
                        whole_step_fp64_equivalent_tflops=value / world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, fl = oracle_sample_tflops()
        cpu = {"value": v, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "seconds": dt,
               "sample": f"oracle column selected inversion, 1 thread, on the {CPU_SAMPLE_SIDE}^3 member of the "
                         f"same grid family ({fl:.3e} algorithmic flops)"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64" if not args.fp64_emulation else "f64 (steps 2, 3: bf16 slice products, exact integer sums)",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": prob.n, "nnz_a_lower": info["nnz_a"],
                           "nnz_l": info["nnz_l"], "supernodes": info["nsn"], "levels": info["nlevels"],
                           "flops_per_step": flops, "schedule": "level (one grouped launch per kernel per level)",
                           "batched_ms": ms, "graph_ms": ms_graph, "persistent_ms": ms_persistent, "plain_ms": ms_plain,
                           "speedup_batched_vs_plain": ms_plain / ms if ms_plain else None,
                           "kernel_ms_per_step": {"normalise": kms[0] / args.steps, "step2_gemm1": kms[1] / args.steps,
                                                  "step3_partials": kms[2] / args.steps,
                                                  "step3_finish": kms[3] / args.steps},
                           "l2": "no flush: the X panels (%.1f GB) exceed L2 (129 MB)" % (info["panel_entries"] * 8 / 1e9),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "fp64_emulation": emul},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(sum(kl)), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_emulation(args, prob, info, vals, h64, stream, dev):
    """LEVEL selinv with opts.fp64_emulation = 1 on the same matrix: time,
    kernel classes, max |X_em - X_fp64| / max |X_fp64| over every X panel
    entry (h64 holds the FP64 selected inverse), and the step-2 class's bf16
    tensor rate (28 slice products per multiply-add of X_{C,C} Lhat)."""
    import torch
    import paper_1404_0447_gb300 as P
    he = P.SelInv(prob.n, prob.colptr, prob.rowind, max_sn_width=128, relax=P.RELAX_AMALG,
                  fp64_emulation=args.emulation_variant, **tuning(args))
    with torch.cuda.stream(stream):
        he.factor(vals, stream=stream)
        for _ in range(max(1, args.warmup - 1)):
            he.selinv(P.LEVEL, stream=stream)
    he.sync_status(stream=stream)
    torch.cuda.synchronize()
    he.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        he.selinv(P.LEVEL, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kms, kl = he.get_timing()
    he.set_timing(False)
    he.sync_status(stream=stream)
    xe, x64 = he.panels(0, stream=stream)[0], h64.panels(0, stream=stream)[0]
    torch.cuda.synchronize()
    diff = float((torch.max(torch.abs(xe - x64)) / torch.max(torch.abs(x64))).item())
    del xe, x64
    # end to end as in the headline's e2e: pinned values in, factor, selinv with
    # the X panels streamed to pinned host memory (second of two runs)
    e2e_ms = None
    if not args.no_e2e:
        host_vals = torch.tensor(prob.values, dtype=torch.float64).pin_memory()
        host_out = torch.empty(info["panel_entries"], dtype=torch.float64).pin_memory()
        dev_vals = torch.empty_like(vals)
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                dev_vals.copy_(host_vals, non_blocking=True)
                he.factor(dev_vals, stream=stream)
                he.selinv_to_host(host_out, stream=stream)
            stream.synchronize()
            e2e_ms = 1e3 * (time.perf_counter() - t0)
        he.sync_status(stream=stream)
    s2_ms = kms[1] / args.steps
    out = {"ms_per_step": ms, "fp64_equivalent_tflops": info["flops_selinv"] / (ms * 1e-3) / 1e12,
           "e2e_ms_per_step": e2e_ms,
           "kernel_ms_per_step": {"normalise": kms[0] / args.steps, "step2_split_and_products": s2_ms,
                                  "step3_split_and_partials": kms[2] / args.steps,
                                  "step3_finish_and_x_split": kms[3] / args.steps},
           "max_rel_diff_vs_fp64_x": diff,
           "step2_roofline": emulated_step2_roofline(info["flops_gemm1"], s2_ms),
           "arithmetic": "steps 2 and 3 on 7 x 8-bit bf16 slices of 2^-(e_p+e_q) X, of diag(2^e_C) Lhat and of "
                         "diag(2^-e_C) X_CK, exact FP32 group sums over 32-row chunks, 64-bit integer "
                         "accumulation; every other step FP64"}
    del he
    return out


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
    line = {"workload": w, "steps": args.steps, "warmup": args.warmup}
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
        line["factor_ms"] = _time(factor, 1, 0, st)
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
        line[f"{name}_frac_of_fp64_peak"] = line[f"{name}_tflops"] / FP64_PEAK_TFLOPS
    if "plain_ms" in line:
        line["speedup_level_vs_plain"] = line["plain_ms"] / line["level_ms"]
    if w == "dg_poles":
        # pole expansion Gamma = sum_l w_l X_l (weights 1/P here) and E(z_l) of Eq. (16)
        wts = np.full(info["batch"], 1.0 / info["batch"], np.complex128)
        gam = torch.empty(info["panel_entries"], dtype=torch.complex128, device=dev)
        line["pole_sum_ms"] = _time(lambda: h.pole_sum(wts, out=gam, stream=st), 3, 1, st)
        line["pole_sum_GBps"] = (info["batch"] + 1) * info["panel_entries"] * 16 / (line["pole_sum_ms"] * 1e-3) / 1e9
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
        line[f"{s2}_frac_of_fp64_peak"] = line[f"{s2}_tflops"] / FP64_PEAK_TFLOPS
    if w == "graphlap48":
        # differentiable logdet: forward = factor + logdet, backward = selinv + gradient gather
        g = torch.empty(info["nnz_a"], dtype=torch.float64, device=dev)
        line["logdet_forward_ms"] = _time(lambda: (h.factor(vals, stream=st), h.logdet(stream=st)), 3, 1, st)
        line["logdet_backward_ms"] = _time(lambda: (h.selinv(P.LEVEL, stream=st), h.logdet_grad(out=g, stream=st)),
                                           args.steps, 1, st)
        G = torch.randn(info["panel_entries"], dtype=torch.float64, device=dev)
        h.selinv(P.LEVEL, stream=st)
        line["adjoint_ms"] = _time(lambda: h.adjoint(G, stream=st), 3, 1, st)
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


# Compute-only throughput probe (no memory traffic in the timed loops):
# independent DFMA chains and back-to-back mma.sync of several shapes on
# register operands.
PEAK_PROBE_CU = r"""
#include <cstdio>
#include <cuda_runtime.h>
__global__ void dfma(double* out, int iters) {
  double x[8];
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-9 + q;
  const double a = 1.0 - 1e-12, c = 1e-13;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, c);
  double s = 0; for (int q = 0; q < 8; ++q) s += x[q];
  if (s == 12345.0) out[threadIdx.x] = s;
}
__global__ void dmma(double* out, int iters) {
  double d[4][2] = {};
  const double a = threadIdx.x * 1e-3, b = threadIdx.x * 2e-3;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d[q][0]), "+d"(d[q][1]) : "d"(a), "d"(b));
  double s = 0; for (int q = 0; q < 4; ++q) s += d[q][0] + d[q][1];
  if (s == 12345.0) out[threadIdx.x] = s;
}
__global__ void hmma_bf16(double* out, int iters) {
  float d[4][4] = {};
  const unsigned a0 = threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u, b0 = a0 * 11u, b1 = a0 * 13u;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(d[q][0]), "+f"(d[q][1]), "+f"(d[q][2]), "+f"(d[q][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  float s = 0; for (int q = 0; q < 4; ++q) for (int i = 0; i < 4; ++i) s += d[q][i];
  if (s == 12345.f) out[threadIdx.x] = s;
}
__global__ void imma_s8(double* out, int iters) {
  int d[4][4] = {};
  const unsigned a0 = threadIdx.x, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u, b0 = a0 * 11u, b1 = a0 * 13u;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+r"(d[q][0]), "+r"(d[q][1]), "+r"(d[q][2]), "+r"(d[q][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  int s = 0; for (int q = 0; q < 4; ++q) for (int i = 0; i < 4; ++i) s += d[q][i];
  if (s == 12345) out[threadIdx.x] = s;
}
int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  double* buf = nullptr;
  cudaMalloc(&buf, 4096 * sizeof(double));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads = 256, blocks = sms * 8;
  const char* names[4] = {"dfma", "dmma_m8n8k4_f64", "mma_sync_m16n8k16_bf16", "mma_sync_m16n8k32_s8"};
  const double flops[4] = {8.0 * 2, 4.0 * 8 * 8 * 4 * 2, 4.0 * 16 * 8 * 16 * 2, 4.0 * 16 * 8 * 32 * 2};
  const double per_thread[4] = {1, 1.0 / 32, 1.0 / 32, 1.0 / 32};  // loop bodies: per thread (DFMA) or per warp (MMA)
  const int iters[4] = {20000, 400, 4000, 1500};
  for (int c = 0; c < 4; ++c) {
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0);
      if (c == 0) dfma<<<blocks, threads>>>(buf, iters[c]);
      if (c == 1) dmma<<<blocks, threads>>>(buf, iters[c]);
      if (c == 2) hmma_bf16<<<blocks, threads>>>(buf, iters[c]);
      if (c == 3) imma_s8<<<blocks, threads>>>(buf, iters[c]);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    const double units = (double)blocks * threads * per_thread[c] * iters[c];
    printf("%s %.4f\n", names[c], units * flops[c] / (ms * 1e-3) / 1e12);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) printf("error %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}
"""


def run_peaks(args):
    """Measured peaks of this GPU: FP64 DFMA and DMMA, bf16 and int8 mma.sync
    (compute-only probe, compiled here with nvcc), and cuBLAS DGEMM through
    torch.matmul on float64 (8192^3, best of 3 after 2 warm-ups)."""
    import subprocess
    import tempfile
    import torch
    out = {"what": "peak probe", "unit": "TFLOP/s (int8: TOP/s)"}
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "peaks.cu")
        exe = os.path.join(d, "peaks")
        with open(src, "w") as f:
            f.write(PEAK_PROBE_CU)
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src])
        for line in subprocess.check_output([exe], text=True).splitlines():
            k, v = line.split()
            out[k] = float(v)
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    bmat = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    best = 1e30
    for it in range(5):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, bmat)
        e1.record()
        e1.synchronize()
        if it >= 2:
            best = min(best, e0.elapsed_time(e1))
    out["cublas_dgemm_8192"] = 2 * 8192 ** 3 / (best * 1e-3) / 1e12
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.peaks:
        run_peaks(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "grid3d_80":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
