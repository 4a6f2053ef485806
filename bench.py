"""Benchmark: condensation log-determinant throughput on GB300 (one JSON line).

A step is one full condensation sweep (stage, every pivot step, finalize) of the
N x N benchmark matrix through liblogdet. Throughput is counted as 2N^3/3 flop
per sweep (TFLOP/s). Inputs: dense iid N(0, 1/N) entries, N = 8000, seed 1,
generated with numpy's default_rng (bit-identical on every host).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode f64_plain]
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
N_DEFAULT = 8000
SEED = 1

# nominal dense tensor rates relative to BF16 (TF32 1.1 / BF16 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
DTYPE = {"f64_plain": "f64", "f32_plain": "f32", "f64_blocked": "f64", "f32_tf32": "f32+tf32",
         "f32_3xtf32": "f32+3xtf32", "f32_bf16x3": "f32+bf16x3"}


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


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(A, target_s=12.0, threads=None):
    """Times the oracle on the host cores over the first S pivot steps of A."""
    import oracle

    N = A.shape[0]
    threads = threads or (os.cpu_count() or 1)
    oracle.build()
    s0 = min(N, 8)
    t0 = time.perf_counter()
    oracle.logdet(A, max_steps=s0, nthreads=threads)
    t_cal = max(time.perf_counter() - t0, 1e-3)
    S = int(max(s0, min(N, s0 * target_s / t_cal)))
    t0 = time.perf_counter()
    oracle.logdet(A, max_steps=S, nthreads=threads)
    dt = time.perf_counter() - t0
    fl = sum(2.0 * (N - s - 1) ** 2 for s in range(S))
    return {"value": fl / dt / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {S} of {N} condensation steps of the N={N} benchmark matrix "
                      f"({fl:.3g} flop in {dt:.2f} s, FP64, {threads} threads)"}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    import workloads
    N = args.N
    A = workloads.dense_gaussian(N, seed=SEED, var=1.0 / N)
    # each step: a bounded sample of the sweep, sized so the whole run takes minutes
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(A, target_s=per_step * 0.3)
    vals = []
    samples = []
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
        "config": {"workload": f"dense iid N(0,1/N) N={N} seed {SEED}, plain FP64 condensation "
                               f"(oracle, host cores)", "N": N, "mode": "f64_plain"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ rooflines
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of the kernel as it stands; keyed by
# (kernel class, workload). Reported only for the workload it was taken on.
NCU_TRAFFIC = {
    ("panel", "dense N=8000 f32_3xtf32"): {
        "bytes": 3868928 + 256,
        "launch": "6th panel of a sweep (m0 = 7360); its declared algorithmic bytes: 67.8e6",
        "summary": "profiles/panel_cluster_kernel_n8000.md"},
    ("batched", "batched4096"): {
        "bytes": 11386784000 + 11559038000,
        "launch": "the whole batch (one launch per step)",
        "summary": "profiles/batched_kernel_spd4096.md"},
}


def make_roofline(kernel, mode, k_bytes, k_flops, k_ms, k_launches, steps):
    peaks = read_peaks()
    sec = k_ms * 1e-3
    out = {"kernel": kernel, "traffic": None, "peak_source": peaks["source"],
           "kernel_ms_per_step": k_ms / steps, "kernel_launches_per_step": k_launches / steps,
           "algorithmic_bytes_per_step": k_bytes / steps,
           "algorithmic_flops_per_step": k_flops / steps}
    if kernel == "rankb_tc":
        # tensor-bound contraction; split modes run 3 products per useful flop
        bf16 = peaks["bf16_tflops_sustained"]
        if mode == "f32_bf16x3":
            peak, note = bf16 / 3.0, "BF16 sustained / 3 (three products)"
        elif mode == "f32_3xtf32":
            peak, note = bf16 * TF32_OVER_BF16 / 3.0, "BF16 sustained x 1.1/2.25 (TF32) / 3"
        else:
            peak, note = bf16 * TF32_OVER_BF16, "BF16 sustained x 1.1/2.25 (TF32)"
        ach = k_flops / sec / 1e12 if sec > 0 else None
        out.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak if ach else None, "peak_note": note})
        hbm = k_bytes / sec / 1e9 if sec > 0 else None
        out["hbm_gbs_same_kernel"] = hbm
    else:
        ach = k_bytes / sec / 1e9 if sec > 0 else None
        peak = peaks["hbm_gbs"]
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak if ach else None})
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


def other_paths(pk, _lib, A, main_mode, dev, err_gold=None):
    """Quick timings of the other paths (each entry independent; errors recorded)."""
    import torch
    import workloads
    res = {}
    N = A.shape[0]
    g = None
    if err_gold and os.path.exists(err_gold):
        with open(err_gold) as f:
            g = json.load(f)
    for mode in ["f64_plain", "f32_plain", "f64_blocked", "f32_tf32", "f32_3xtf32", "f32_bf16x3"]:
        if mode == main_mode:
            continue
        try:
            steps = 1 if mode in ("f64_plain", "f32_plain", "f64_blocked") else 3
            ms, (sg, la) = time_call(lambda: pk.logdet(A, mode), 1, steps, dev)
            e = {"ms_per_sweep": ms, "tflops": flops(N) / (ms * 1e-3) / 1e12}
            if g:
                e["rel_err_vs_oracle"] = abs(float(la) - g["logabs"]) / max(1.0, abs(g["logabs"]))
                e["sign_match"] = float(sg) == g["sign"]
            res[mode] = e
        except Exception as ex:  # report, do not fail the benchmark line
            res[mode] = {"error": str(ex)[:200]}
    try:
        sizes = workloads.batched_sizes(4096, seed=3)
        mats = workloads.batched_covariances_torch(sizes, seed=3, device=dev)
        batch = pk.BatchedInputs(mats)
        ms, _ = time_call(lambda: pk.logdet_batched(batch, "f32_plain"), 2, 5, dev)
        fl = float(sum(2.0 * int(n) ** 3 / 3.0 for n in sizes))
        res["batched_4096_f32"] = {"ms": ms, "dets_per_s": 4096 / (ms * 1e-3),
                                   "tflops": fl / (ms * 1e-3) / 1e12,
                                   "workload": "4096 SPD X^T X/(2n)+1e-2 I, n uniform on "
                                               "{32,...,512}, seed 3, FP32, one launch"}
        del mats, batch
    except Exception as ex:
        res["batched_4096_f32"] = {"error": str(ex)[:200]}
    try:
        B, n = 256, 1024
        gen = torch.Generator(device=dev).manual_seed(4)
        lam = 10.0 ** (-2.0 * torch.rand(B, n, generator=gen, device=dev, dtype=torch.float64))
        Q, R = torch.linalg.qr(torch.randn(B, n, n, generator=gen, device=dev, dtype=torch.float64))
        Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
        X = ((Q * lam[:, None, :]) @ Q.transpose(1, 2)).float()
        del Q, R

        for gm in ("f32_3xtf32", "f32_plain"):
            def fb():
                Xg = X.detach().requires_grad_(True)
                out = pk.logabsdet(Xg, gm)
                out.sum().backward()
                return Xg.grad
            ms, _ = time_call(fb, 1, 2, dev)
            res[f"grad_256x1024_{gm}"] = {"ms_forward_backward": ms,
                                          "fwd_bwd_tflops": (B * (2 * n ** 3 / 3 + 2 * n ** 3)) /
                                          (ms * 1e-3) / 1e12}
    except Exception as ex:
        res["grad_256x1024"] = {"error": str(ex)[:200]}
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
    import workloads

    N = args.N
    mode = args.mode
    stream = torch.cuda.current_stream(dev)
    if args.workload != "dense":
        return run_other_workload(args, pk, _lib, dev, stream, rank, world)
    A_np = workloads.dense_gaussian(N, seed=SEED, var=1.0 / N)
    A = torch.from_numpy(A_np).to(dev)

    def step():
        return pk.logdet(A, mode)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        sg, la = step()
    barrier()

    # accuracy of this result against the stored FP64 oracle value
    err = None
    gold = os.path.join(ROOT, "tests", "golden", f"oracle_dense_n{N}_seed{SEED}.json")
    if os.path.exists(gold):
        with open(gold) as f:
            g = json.load(f)
        err = {"logabs": float(la), "oracle_logabs": g["logabs"],
               "rel_err": abs(float(la) - g["logabs"]) / max(1.0, abs(g["logabs"])),
               "sign_match": float(sg) == g["sign"]}

    # one fully profiled sweep: per-class shares, then the dominant class
    _lib.ld_profile_start(None)
    step()
    torch.cuda.synchronize(dev)
    _lib.ld_profile_stop()
    shares = {}
    for cls in _lib.ld_profile_classes():
        nl, tms = _lib.ld_profile_query(cls)
        shares[cls] = {"launches": nl, "ms": round(tms, 4)}
    tot = sum(v["ms"] for v in shares.values()) or 1.0
    for v in shares.values():
        v["share"] = round(v["ms"] / tot, 4)
    kernel = max(shares, key=lambda k: shares[k]["ms"]) if shares else "update"
    # the tensor-core trailing update of the same profiled sweep (its own event time)
    tc_work = _lib.ld_profile_work("rankb_tc") if "rankb_tc" in shares else None
    clocks = ClockSampler(local)
    time.sleep(0.3)
    _lib.ld_profile_start(kernel)
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
    k_launches, k_ms = _lib.ld_profile_query(kernel)

    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t[0])
    value = world * flops(N) / (ms_max * 1e-3) / 1e12

    # roofline of the dominant kernel: algorithmic work over its event time
    k_bytes, k_flops = _lib.ld_profile_work(kernel)
    roofline = make_roofline(kernel, mode, k_bytes, k_flops, k_ms, k_launches, args.steps)
    tr = NCU_TRAFFIC.get((kernel, f"dense N={N} {mode}"))
    if tr:
        roofline["traffic"] = tr["bytes"]
        roofline["traffic_note"] = f"ncu, one launch: {tr['launch']} ({tr['summary']})"
    if kernel == "panel":
        # the panel is a serial chain of pivots: its time per pivot is the figure to cut
        roofline["pivot_chain"] = {"pivots_per_step": N,
                                   "us_per_pivot": 1e3 * k_ms / args.steps / N}
    if tc_work and kernel != "rankb_tc":
        roofline["secondary"] = make_roofline("rankb_tc", mode, tc_work[0], tc_work[1],
                                              shares["rankb_tc"]["ms"],
                                              shares["rankb_tc"]["launches"], 1)
    roofline["kernel_shares"] = shares

    # end to end: pinned host input -> device -> sweep -> host result, per step
    A_host = torch.from_numpy(A_np).pin_memory()
    A_dev = torch.empty_like(A)
    import ctypes
    hs, hl = ctypes.c_double(), ctypes.c_double()
    mcode = _lib.MODES[mode]
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A_dev.copy_(A_host, non_blocking=True)
        code = _lib.ld_logdet(A_dev.data_ptr(), _lib.LD_DTYPE_F64, N, N, mcode,
                              stream.cuda_stream, ctypes.addressof(hs), ctypes.addressof(hl))
        _lib.check("ld_logdet", code)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": world * flops(N) / float(te[0]) / 1e12, "unit": UNIT,
           "h2d_bytes_per_step": A_np.nbytes, "d2h_bytes_per_step": 16}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(A_np, target_s=args.cpu_seconds)
    paths = None
    if rank == 0 and not args.no_paths:
        paths = other_paths(pk, _lib, A, mode, dev, err_gold=gold)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE.get(mode, mode), "data": "synthetic",
            "config": {"workload": f"dense iid N(0,1/N) N={N} seed {SEED}, one sweep per step",
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


def run_other_workload(args, pk, _lib, dev, stream, rank, world):
    """The batched (4096 covariance matrices) and gradient (256 x 1024^2) workloads
    as their own benchmark line (units: dets/s and matrices/s)."""
    import torch
    import torch.distributed as dist
    import workloads
    if args.workload == "batched4096":
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
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    _lib.ld_profile_start(None)
    step()
    torch.cuda.synchronize(dev)
    _lib.ld_profile_stop()
    shares = {}
    for cls in _lib.ld_profile_classes():
        nl, tms = _lib.ld_profile_query(cls)
        shares[cls] = {"launches": nl, "ms": round(tms, 4)}
    tc_work = None
    if args.workload != "batched4096" and shares:
        # the roofline follows the kernel with the largest share; the tensor-core
        # update (same profiled step, its own event time) is reported beside it
        kernel = max(shares, key=lambda k: shares[k]["ms"])
        if "rankb_tc" in shares and kernel != "rankb_tc":
            tc_work = _lib.ld_profile_work("rankb_tc")
    clocks = ClockSampler(dev.index or 0)
    _lib.ld_profile_start(kernel)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # under torchrun every rank sweeps its own batch (weak scaling, no collective
    # on the data path); the job's time is the slowest rank's
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    _lib.ld_profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        tm = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms = float(tm[0])
    launches_all, _ = _lib.ld_profile_query(None)
    k_launches, k_ms = _lib.ld_profile_query(kernel)
    peaks = read_peaks()
    # the FP32 SIMT FMA peak: 152 SMs x 128 FMA/clk x 2 flop at the sampled SM clock
    sm_mhz = clk.get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    k_flop = flop * args.steps if args.workload == "batched4096" else None
    roof = None
    if args.workload != "batched4096" and k_ms > 0:
        kb, kf = _lib.ld_profile_work(kernel)
        roof = make_roofline(kernel, "f32_3xtf32", kb, kf, k_ms, k_launches, args.steps)
        if tc_work:
            roof["secondary"] = make_roofline("rankb_tc", "f32_3xtf32", tc_work[0], tc_work[1],
                                              shares["rankb_tc"]["ms"],
                                              shares["rankb_tc"]["launches"], 1)
        roof["kernel_shares"] = shares
    if k_flop and k_ms > 0:
        ach = k_flop / (k_ms * 1e-3) / 1e12
        roof = {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": ach / alu_peak,
                "traffic": NCU_TRAFFIC[("batched", "batched4096")]["bytes"],
                "traffic_note": "ncu, one launch: " + NCU_TRAFFIC[("batched", "batched4096")]["launch"],
                "peak_note": "FP32 FMA: SMs x 128 lanes x 2 flop x sampled SM clock",
                "kernel_shares": shares}
    value = world * units / (ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl, "l2": "inputs larger than L2"},
            "roofline": roof or {"kernel_shares": shares}, "tflops": flop / (ms * 1e-3) / 1e12,
            "gpu_launches": launches_all, "clocks": clk, "cpu_baseline": None,
            "e2e": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="f32_3xtf32")
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paths", action="store_true")
    ap.add_argument("--workload", default="dense", choices=["dense", "batched4096", "grad256x1024"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
