"""Benchmark: condensation log-determinant throughput on GB300 (one JSON line).

A step is one full condensation sweep (stage, every pivot step, finalize) of the
N x N benchmark matrix through liblogdet; throughput is counted as 2N^3/3 flop
per sweep (TFLOP/s). The default line is the largest single-GPU workload:
N = 32768, A = Q diag(lambda) Q^T with Q Haar (QR of a Gaussian) and lambda
log-uniform in [1e-4, 1] (seed 2), stored in FP32, swept with the trailing update
in split TF32 (3xTF32); its error is taken against the exact sum of log(lambda).
Every other workload (N = 16384 of the same recipe, the N = 8000 iid and
covariance matrices in every mode, the 4096-matrix batch and the 256-matrix
gradient) is measured beside it under "paths", each with its error and roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode f32_3xtf32]
                    [--workload spd32768|spd16384|dense|spdcov8000|batched4096|grad256x1024]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

With N > 1 (torchrun), every rank runs an independent replica of the sweep (a
single matrix does not shard) and the value is the whole job's throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logdet TFLOP/s (2N³/3) and batched dets/s, mixed vs plain FP64 at stated error"
UNIT = "TFLOP/s"

# nominal dense tensor rates relative to BF16 (TF32 1.1 / BF16 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
DTYPE = {"f64_plain": "f64", "f32_plain": "f32", "f64_blocked": "f64", "f32_tf32": "f32+tf32",
         "f32_3xtf32": "f32+3xtf32", "f32_bf16x3": "f32+bf16x3", "f64_ozaki": "f64+bf16 slices"}
TENSOR_MODES = ("f32_tf32", "f32_3xtf32", "f32_bf16x3", "f64_ozaki")
ALL_MODES = ["f64_plain", "f32_plain", "f64_blocked", "f64_ozaki", "f32_tf32", "f32_3xtf32",
             "f32_bf16x3"]
# slice products of the FP64-accurate update per useful product (orders 0..5 of six slices)
OZAKI_PRODUCTS = 21

# single-matrix workloads: (N, description)
WORKLOADS = {
    "spd32768": (32768, "SPD Q diag(lambda) Q^T, Q Haar, lambda log-uniform [1e-4,1], seed 2, "
                        "N=32768, FP32 storage; error vs exact sum log(lambda)"),
    "spd16384": (16384, "SPD Q diag(lambda) Q^T, Q Haar, lambda log-uniform [1e-4,1], seed 2, "
                        "N=16384, FP32 storage; error vs exact sum log(lambda)"),
    "dense": (8000, "dense iid N(0,1/N), seed 1; error vs the stored FP64 oracle result"),
    "spdcov8000": (8000, "SPD X^T X/(2N)+1e-3 I, X 2N x N iid N(0,1) drawn after the dense "
                         "matrix of seed 1, N=8000; error vs the stored FP64 oracle result"),
}


def flops(N):
    return 2.0 * N ** 3 / 3.0


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


def tensor_peak(mode, peaks=None):
    """Dense tensor peak of the trailing update's arithmetic, in useful (FP32-
    equivalent) TFLOP/s: the measured sustained BF16 rate, times the nominal
    TF32/BF16 ratio for TF32, divided by the three products of the split kinds."""
    peaks = peaks or read_peaks()
    bf16 = peaks["bf16_tflops_sustained"]
    if mode == "f64_ozaki":
        return (bf16 / OZAKI_PRODUCTS,
                f"BF16 sustained / {OZAKI_PRODUCTS} (slice products per FP64 product)")
    if mode == "f32_bf16x3":
        return bf16 / 3.0, "BF16 sustained / 3 (three products)"
    if mode == "f32_3xtf32":
        return bf16 * TF32_OVER_BF16 / 3.0, "BF16 sustained x 1.1/2.25 (TF32) / 3"
    return bf16 * TF32_OVER_BF16, "BF16 sustained x 1.1/2.25 (TF32)"


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.err = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", sel],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:  # no nvidia-smi: report why
            self.err = str(e)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": self.err}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ inputs
def make_input(workload, N, dev):
    """(A on dev, reference logabs, reference sign, reference note). The SPD
    recipes are generated on the GPU in FP64 and stored in FP32; the iid and
    covariance matrices on the host in FP64 (numpy default_rng)."""
    import torch
    import workloads
    if workload in ("spd32768", "spd16384"):
        A, sl = workloads.spd_haar_torch(N, seed=2, lo=1e-4, hi=1.0, device=dev,
                                         dtype=torch.float32)
        return A, sl, 1.0, "exact sum of log(lambda)"
    if workload == "dense":
        A = torch.from_numpy(workloads.dense_gaussian(N, seed=1, var=1.0 / N)).to(dev)
        gold = os.path.join(ROOT, "tests", "golden", f"oracle_dense_n{N}_seed1.json")
    else:
        A = torch.from_numpy(workloads.dense_and_spd_pair(N, seed=1)[1]).to(dev)
        gold = os.path.join(ROOT, "tests", "golden", f"oracle_spd_n{N}_seed1.json")
    if os.path.exists(gold):
        with open(gold) as f:
            g = json.load(f)
        return A, g["logabs"], g["sign"], "stored FP64 oracle result"
    return A, None, None, None


def accuracy(sg, la, ref, ref_sign):
    if ref is None:
        return None
    return {"logabs": float(la), "ref_logabs": ref,
            "rel_err": abs(float(la) - ref) / max(1.0, abs(ref)),
            "sign_match": float(sg) == ref_sign}


# ------------------------------------------------------------------ CPU oracle
_ORACLE_CAL = {}


def oracle_sample(A, target_s=12.0, threads=None, what="benchmark matrix"):
    """Times the oracle on the host cores over the first S pivot steps of A (S
    sized for about target_s seconds of steps). The time is the difference of a
    run of S steps and a run of none, so the oracle's one-off copy of A into its
    working matrix is not counted against the steps. The per-step estimate that
    sizes S is taken once per matrix (the first steps are the dearest, so later
    steps only shorten the sample)."""
    import oracle

    N = A.shape[0]
    threads = threads or (os.cpu_count() or 1)
    oracle.build()

    def run(steps):
        t0 = time.perf_counter()
        oracle.logdet(A, max_steps=steps, nthreads=threads)
        return time.perf_counter() - t0

    key = (id(A), N, threads)
    if key not in _ORACLE_CAL:
        t0 = run(0)
        s_b = min(N, 8)
        while True:  # a difference well above the run-to-run noise of the copy
            d = run(s_b) - t0
            if d >= 0.5 or s_b >= N:
                break
            s_b = min(N, 4 * s_b)
        _ORACLE_CAL[key] = max(d / max(1, s_b), 1e-6)
    per_step = _ORACLE_CAL[key]
    S = int(max(1, min(N, target_s / per_step)))
    t0 = run(0)
    dt = max(run(S) - t0, 1e-9)
    fl = sum(2.0 * (N - s - 1) ** 2 for s in range(S))
    share = fl / flops(N)
    return {"value": fl / dt / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {S} of the {N} condensation steps of the N={N} {what} "
                      f"({fl:.3g} flop in {dt:.2f} s: a run of {S} steps minus a run of none, "
                      f"so the copy of A is not counted; {100 * share:.1f}% of the sweep's "
                      f"flops; FP64, {threads} threads)"}


def oracle_full_sweep(A, threads=None, what="matrix"):
    """Times one whole oracle sweep of A on the host cores."""
    import oracle

    N = A.shape[0]
    threads = threads or (os.cpu_count() or 1)
    oracle.build()
    t0 = time.perf_counter()
    oracle.logdet(A, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": flops(N) / dt / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
            "seconds": dt, "sample": f"the whole sweep of the N={N} {what} (FP64, {threads} threads)"}


def host_matrix(workload, N):
    """The workload's matrix on the host in FP64 (for the oracle)."""
    import numpy as np
    import workloads
    if workload == "dense":
        return workloads.dense_gaussian(N, seed=1, var=1.0 / N)
    if workload == "spdcov8000":
        return workloads.dense_and_spd_pair(N, seed=1)[1]
    import torch
    A, _ = workloads.spd_haar_torch(N, seed=2, lo=1e-4, hi=1.0, device="cuda",
                                    dtype=torch.float32)
    out = A.cpu().double().numpy()
    del A
    torch.cuda.empty_cache()
    return np.ascontiguousarray(out)


def run_reference(args):
    """The oracle on the host cores, on bounded samples of this benchmark's workload."""
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    N = args.N or WORKLOADS[args.workload][0]
    A = host_matrix(args.workload, N)
    # each step: a bounded sample of the sweep, sized so the whole run takes minutes
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(A, target_s=per_step * 0.3)
    vals, samples = [], []
    for _ in range(args.steps):
        cb = oracle_sample(A, target_s=per_step)
        vals.append(cb["value"])
        samples.append(cb)
    v = statistics.median(vals)
    cb = dict(samples[-1])
    cb["value"] = v
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": flops(N) / (v * 1e12) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1] +
                   ", plain FP64 condensation (oracle, host cores)", "N": N, "mode": "f64_plain"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ rooflines
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel, from one ncu capture of the kernel as it stands; keyed by (kernel
# class, workload). Reported only for the workload it was taken on.
NCU_TRAFFIC = {
    ("batched", "batched4096"): {
        "bytes": 11523763712 + 11589309952,
        "launch": "the whole batch (one launch per step)",
        "summary": "profiles/batched_kernel_spd4096.md"},
}
# Measured DRAM bytes over algorithmic bytes of a kernel class across a whole
# sweep (every launch of one step captured), for kernels whose launches at the
# benchmark's size are too many or too large to capture: the per-launch traffic
# at any size is this ratio times the launch's algorithmic bytes (the traffic of
# the tensor-core update grows with the D bytes it moves). Keyed by (kernel
# class, mode).
NCU_TRAFFIC_RATIO = {
    ("rankb_tc", "f32_3xtf32"): {
        "ratio": (30959057152 + 20334375680) / 50070683648.0,
        "captured": "all 314 launches of one N=16384 SPD sweep (3xTF32)",
        "summary": "profiles/rankb_tc_traffic_3xtf32_spd16384.md"},
}


def make_roofline(kernel, mode, k_bytes, k_flops, k_ms, k_launches, steps):
    """Roofline of one kernel class: its algorithmic work over its summed event
    time. The tensor-core update is tensor-bound; the others are reported against
    HBM."""
    peaks = read_peaks()
    sec = k_ms * 1e-3
    out = {"kernel": kernel, "traffic": None, "peak_source": peaks["source"],
           "kernel_ms_per_step": k_ms / steps, "kernel_launches_per_step": k_launches / steps,
           "algorithmic_bytes_per_step": k_bytes / steps,
           "algorithmic_flops_per_step": k_flops / steps}
    if kernel in ("rankb_tc", "rankb_ozaki"):
        tr = NCU_TRAFFIC_RATIO.get((kernel, mode))
        if tr and k_launches > 0:
            out["traffic"] = tr["ratio"] * k_bytes / k_launches
            out["traffic_note"] = (f"per launch: {tr['ratio']:.3f} x the launch's algorithmic "
                                   f"bytes, the ratio measured by ncu over {tr['captured']}")
        peak, note = tensor_peak(mode, peaks)
        ach = k_flops / sec / 1e12 if sec > 0 else None
        out.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak if ach else None, "peak_note": note})
        out["hbm_gbs_same_kernel"] = k_bytes / sec / 1e9 if sec > 0 else None
    else:
        ach = k_bytes / sec / 1e9 if sec > 0 else None
        peak = peaks["hbm_gbs"]
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak if ach else None})
    return out


def profile_step(_lib, step, dev):
    """Per-class launches, event time and declared work of one step. A first
    pass counts every class's launches and work without events; then each class
    is timed in steps of its own, once pipelined and once with the sweep on one
    stream (events around that class's launches only: with every launch of the
    concurrent streams bracketed at once, the summed spans came out tens of times
    longer than the step). The dominant kernel's own roofline is timed again over
    the timed region."""
    import torch

    def one(filt):
        _lib.ld_profile_start(filt)
        step()
        torch.cuda.synchronize(dev)
        _lib.ld_profile_stop()

    one("\x01")  # a class name no launch has: counts and work only
    shares = {}
    for cls in _lib.ld_profile_classes():
        nl, _ = _lib.ld_profile_query(cls)
        b, f = _lib.ld_profile_work(cls)
        shares[cls] = {"launches": nl, "ms": 0.0, "bytes": b, "flops": f}
    # "ms": the class's summed spans in the pipelined sweep (what the rooflines
    # use); "ms_serial" and "share": the same with the sweep on one stream, one
    # launch after another, comparable with a profiler's launch list (on the
    # overlapped low-priority streams a span also counts the wait for SMs)
    for cls in shares:
        one(cls)
        shares[cls]["ms"] = round(_lib.ld_profile_query(cls)[1], 4)
    old = _lib.ld_get_tuning("sweep_pipeline")
    _lib.ld_set_tuning("sweep_pipeline", 0)
    try:
        for cls in shares:
            one(cls)
            shares[cls]["ms_serial"] = round(_lib.ld_profile_query(cls)[1], 4)
    finally:
        _lib.ld_set_tuning("sweep_pipeline", old)
    tot = sum(v["ms_serial"] for v in shares.values()) or 1.0
    for v in shares.values():
        v["share"] = round(v["ms_serial"] / tot, 4)
    return shares


def sweep_roofline(mode, N, ms, shares):
    """The sweep-level figure: 2N^3/3 useful flop per sweep over the sweep's time,
    against the tensor peak of the update's arithmetic (tensor-core modes), plus
    the tensor-core update's own roofline and the panel chain's time per pivot.
    Plain modes: the rank-1 update kernel against HBM."""
    peaks = read_peaks()
    out = {}
    if mode in TENSOR_MODES:
        peak, note = tensor_peak(mode, peaks)
        ach = flops(N) / (ms * 1e-3) / 1e12
        out = {"kernel": "whole sweep (all kernels, one step)", "bound": "tensor",
               "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "peak_note": note + " (measured sustained BF16; peak_source " + peaks["source"] + ")",
               "traffic": None,
               "traffic_note": "a whole sweep is many launches; the DRAM bytes per launch of its "
                               "dominant kernel are under tensor_update"}
        upd = "rankb_ozaki" if mode == "f64_ozaki" else "rankb_tc"
        if upd in shares:
            s = shares[upd]
            out["tensor_update"] = make_roofline(upd, mode, s["bytes"], s["flops"], s["ms"],
                                                 s["launches"], 1)
    elif mode == "f64_blocked":
        ach = flops(N) / (ms * 1e-3) / 1e12
        out = {"kernel": "whole sweep (all kernels, one step)", "bound": "fp64",
               "achieved": ach, "unit": "TFLOP/s", "peak": None, "frac": None,
               "peak_note": "the FP64 FMA rate of this GPU is not in the measured peaks"}
    if "panel" in shares:
        out["pivot_chain"] = {"pivots_per_step": N, "panel_ms": shares["panel"]["ms"],
                              "us_per_pivot": 1e3 * shares["panel"]["ms"] / N}
    if "update" in shares:
        s = shares["update"]
        upd = make_roofline("update", mode, s["bytes"], s["flops"], s["ms"], s["launches"], 1)
        if not out:
            out = upd
        else:
            out["rank1_update"] = upd
    out["kernel_shares"] = {k: {"launches": v["launches"], "ms": v["ms"],
                                "ms_serial": v.get("ms_serial"), "share": v["share"]}
                            for k, v in shares.items()}
    return out


def time_call(fn, warmup, steps, dev):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        r = fn()
    e1.record()
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps, r


def measure_path(pk, _lib, A, mode, ref, ref_sign, dev, steps=2):
    """Time, error and roofline of one sweep mode on one matrix."""
    N = A.shape[0]
    ms, (sg, la) = time_call(lambda: pk.logdet(A, mode), 1, steps, dev)
    shares = profile_step(_lib, lambda: pk.logdet(A, mode), dev)
    e = {"ms_per_sweep": ms, "tflops": flops(N) / (ms * 1e-3) / 1e12,
         "roofline": sweep_roofline(mode, N, ms, shares)}
    acc = accuracy(sg, la, ref, ref_sign)
    if acc:
        e["rel_err"] = acc["rel_err"]
        e["sign_match"] = acc["sign_match"]
    return e


def other_paths(pk, _lib, dev, main_workload, main_mode, A_main, ref_main):
    """Every other config of the benchmark, each entry independent (errors are
    recorded, not raised)."""
    import torch
    import workloads
    res = {}
    # the headline matrix in its other tensor-core modes
    for mode in TENSOR_MODES:
        if mode == main_mode:
            continue
        try:
            res[f"{main_workload}_{mode}"] = measure_path(pk, _lib, A_main, mode, ref_main, 1.0, dev)
        except Exception as ex:
            res[f"{main_workload}_{mode}"] = {"error": str(ex)[:200]}
    # the other single-matrix configs
    for wl, modes in (("spd16384", TENSOR_MODES), ("dense", ALL_MODES), ("spdcov8000", ALL_MODES)):
        if wl == main_workload:
            continue
        try:
            N = WORKLOADS[wl][0]
            A, ref, ref_sign, note = make_input(wl, N, dev)
            for mode in modes:
                try:
                    steps = 1 if mode in ("f64_plain", "f32_plain", "f64_blocked") else 2
                    e = measure_path(pk, _lib, A, mode, ref, ref_sign, dev, steps=steps)
                    e["workload"] = WORKLOADS[wl][1]
                    res[f"{wl}_{mode}"] = e
                except Exception as ex:
                    res[f"{wl}_{mode}"] = {"error": str(ex)[:200]}
            del A
            torch.cuda.empty_cache()
        except Exception as ex:
            res[wl] = {"error": str(ex)[:200]}
    # the batch and the gradient workloads (their own lines with --workload)
    for wl in ("batched4096", "grad256x1024"):
        try:
            res[wl] = other_workload_line(wl, pk, _lib, dev, 2, 5)
        except Exception as ex:
            res[wl] = {"error": str(ex)[:200]}
    return res


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, local, world = env_rank()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1811_08057_gb300 as pk
    from paper_1811_08057_gb300 import _lib

    stream = torch.cuda.current_stream(dev)
    if args.workload in ("batched4096", "grad256x1024"):
        line = other_workload_line(args.workload, pk, _lib, dev, args.warmup, args.steps,
                                   world=world, full=True)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0

    N = args.N or WORKLOADS[args.workload][0]
    mode = args.mode
    A, ref, ref_sign, ref_note = make_input(args.workload, N, dev)
    torch.cuda.synchronize(dev)

    def step():
        return pk.logdet(A, mode)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        sg, la = step()
    barrier()
    err = accuracy(sg, la, ref, ref_sign)
    if err:
        err["reference"] = ref_note

    # one fully profiled sweep: per-class launches, time and declared work
    shares = profile_step(_lib, step, dev)
    dominant = max(shares, key=lambda k: shares[k]["ms"]) if shares else None

    clocks = ClockSampler(local)
    time.sleep(0.3)
    # inside the timed region only the dominant kernel's launches carry events
    # (every launch is still counted)
    _lib.ld_profile_start(dominant)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sg, la = step()
    e1.record(stream)
    barrier()
    _lib.ld_profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches_all, _ = _lib.ld_profile_query(None)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t[0])
    value = world * flops(N) / (ms_max * 1e-3) / 1e12

    # the sweep-level roofline (class shares from the profiled step); the
    # dominant kernel's figures from its events over the timed region
    if dominant:
        k_launches, k_ms = _lib.ld_profile_query(dominant)
        k_bytes, k_flops = _lib.ld_profile_work(dominant)
        shares[dominant].update({"launches": k_launches / args.steps, "ms": k_ms / args.steps,
                                 "bytes": k_bytes / args.steps, "flops": k_flops / args.steps,
                                 "timed_region": True})
    roofline = sweep_roofline(mode, N, ms_max, shares)
    roofline["dominant_kernel"] = dominant

    # end to end: pinned host input -> device -> sweep -> host result, per step
    import ctypes
    A_host = A.cpu().pin_memory()
    A_dev = torch.empty_like(A)
    hs, hl = ctypes.c_double(), ctypes.c_double()
    mcode = _lib.MODES[mode]
    dcode = _lib.LD_DTYPE_F64 if A.dtype == torch.float64 else _lib.LD_DTYPE_F32
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A_dev.copy_(A_host, non_blocking=True)
        code = _lib.ld_logdet(A_dev.data_ptr(), dcode, N, N, mcode, stream.cuda_stream,
                              ctypes.addressof(hs), ctypes.addressof(hl))
        _lib.check("ld_logdet", code)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": world * flops(N) / float(te[0]) / 1e12, "unit": UNIT,
           "h2d_bytes_per_step": A_host.numel() * A_host.element_size(), "d2h_bytes_per_step": 16}
    del A_host, A_dev

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            A_np = host_matrix(args.workload, N) if args.workload in ("dense", "spdcov8000") \
                else A.cpu().double().numpy()
            cpu = oracle_sample(A_np, target_s=args.cpu_seconds,
                                what=WORKLOADS[args.workload][1].split(";")[0])
            del A_np
            if N > 8000:
                import workloads
                cpu["full_sweep_n8000"] = oracle_full_sweep(
                    workloads.dense_gaussian(8000, seed=1, var=1.0 / 8000),
                    what="dense iid N(0,1/N) matrix of seed 1 (context: a whole sweep)")
        except Exception as ex:
            cpu = {"error": str(ex)[:200]}
    paths = None
    if rank == 0 and not args.no_paths:
        paths = other_paths(pk, _lib, dev, args.workload, mode, A, ref)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE.get(mode, mode), "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1] + ", one sweep per step",
                       "N": N, "mode": mode, "parallelism": "replicas" if world > 1 else "1 gpu",
                       "l2": "inputs larger than L2 (N^2 elements > 129 MB)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_all, "clocks": clk,
            "accuracy": err, "paths": paths,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def other_workload_line(workload, pk, _lib, dev, warmup, steps, world=1, full=False):
    """The batched (4096 covariance matrices) and gradient (256 x 1024^2)
    workloads (units: dets/s and matrices/s), with their own rooflines."""
    import torch
    import torch.distributed as dist
    import workloads
    if workload == "batched4096":
        sizes = workloads.batched_sizes(4096, seed=3)
        mats = workloads.batched_covariances_torch(sizes, seed=3, device=dev)
        batch = pk.BatchedInputs(mats)
        out = (torch.empty(4096, dtype=torch.float64, device=dev),
               torch.empty(4096, dtype=torch.float64, device=dev))

        def step():
            return pk.logdet_batched(batch, "f32_plain", out=out)
        units, unit, kernel = 4096.0, "dets/s", "batched"
        wl = ("4096 SPD X^T X/(2n)+1e-2 I, n uniform on {32,...,512}, seed 3, FP32, "
              "one persistent launch per step")
        flop = float(sum(2.0 * int(n) ** 3 / 3.0 for n in sizes))
    else:
        B, n = 256, 1024
        g = torch.Generator(device=dev).manual_seed(4)
        lam = 10.0 ** (-2.0 * torch.rand(B, n, generator=g, device=dev, dtype=torch.float64))
        Q, R = torch.linalg.qr(torch.randn(B, n, n, generator=g, device=dev, dtype=torch.float64))
        Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
        X = ((Q * lam[:, None, :]) @ Q.transpose(1, 2)).float()
        del Q, R

        def step():
            Xg = X.detach().requires_grad_(True)
            y = pk.logabsdet(Xg, "f32_3xtf32")
            y.sum().backward()
            return Xg.grad
        units, unit, kernel = float(B), "matrices/s", "rankb_tc"
        wl = ("256 SPD 1024x1024 FP32, eigenvalues log-uniform in [1e-2,1], seed 4: log|det| "
              "(batched blocked sweep, 3xTF32) + gradient")
        flop = B * (2.0 * n ** 3 / 3.0 + 2.0 * n ** 3)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    shares = profile_step(_lib, step, dev)
    if workload != "batched4096" and shares:
        kernel = max(shares, key=lambda k: shares[k]["ms"])
    clocks = ClockSampler(dev.index or 0)
    _lib.ld_profile_start(kernel)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # under torchrun every rank sweeps its own batch (weak scaling, no collective
    # on the data path); the job's time is the slowest rank's
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    _lib.ld_profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    if world > 1:
        tm = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms = float(tm[0])
    launches_all, _ = _lib.ld_profile_query(None)
    k_launches, k_ms = _lib.ld_profile_query(kernel)
    roof = None
    if workload == "batched4096" and k_ms > 0:
        # the FP32 SIMT FMA peak: SMs x 128 FMA/clk x 2 flop at the sampled SM clock
        sm_mhz = clk.get("sm_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = flop * steps / (k_ms * 1e-3) / 1e12
        tr = NCU_TRAFFIC.get(("batched", "batched4096"))
        roof = {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": ach / alu_peak,
                "traffic": tr["bytes"] if tr else None,
                "traffic_note": ("ncu, one launch: " + tr["launch"]) if tr else None,
                "peak_note": "FP32 FMA: SMs x 128 lanes x 2 flop x sampled SM clock"}
    elif k_ms > 0:
        kb, kf = _lib.ld_profile_work(kernel)
        roof = make_roofline(kernel, "f32_3xtf32", kb, kf, k_ms, k_launches, steps)
        if "rankb_tc" in shares and kernel != "rankb_tc":
            s = shares["rankb_tc"]
            roof["tensor_update"] = make_roofline("rankb_tc", "f32_3xtf32", s["bytes"], s["flops"],
                                                  s["ms"], s["launches"], 1)
    if roof is not None:
        roof["kernel_shares"] = {k: {"launches": v["launches"], "ms": v["ms"],
                                     "ms_serial": v.get("ms_serial"), "share": v["share"]}
                                 for k, v in shares.items()}
    value = world * units / (ms * 1e-3)
    res = {"value": value, "unit": unit, "ms_per_step": ms, "tflops": flop / (ms * 1e-3) / 1e12,
           "workload": wl, "roofline": roof or {"kernel_shares": shares}}
    if workload == "batched4096":
        res["dets_per_s"] = value
    if not full:
        return res
    return {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "l2": "inputs larger than L2"},
            "roofline": res["roofline"], "tflops": res["tflops"],
            "gpu_launches": launches_all, "clocks": clk, "cpu_baseline": None, "e2e": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="f32_3xtf32")
    ap.add_argument("--workload", default="spd32768",
                    choices=sorted(WORKLOADS) + ["batched4096", "grad256x1024"])
    ap.add_argument("--N", type=int, default=None, help="size (dense workload only)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paths", action="store_true")
    args = ap.parse_args()
    if args.N is not None and args.workload != "dense":
        ap.error("--N applies to the dense workload only")
    if args.impl == "reference":
        if args.workload in ("batched4096", "grad256x1024"):
            ap.error("the reference arm times the single-matrix workloads")
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
