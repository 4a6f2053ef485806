"""The benchmark's reference arm (the oracle on the host cores) on a small matrix:
one JSON line with the keys the benchmark contract asks for. Needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
         "dense", "--N", "256", "--steps", "1", "--warmup", "0"],
        cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "TFLOP/s"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "condensation steps" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_arithmetic():
    """achieved = algorithmic work / event time; peak from the measured peaks
    (3xTF32: BF16 sustained x 1.1/2.25 / 3); frac = achieved / peak."""
    b = _bench_module()
    peaks = b.read_peaks()
    # a tensor-bound launch: 1e12 flop and 1e9 bytes in 10 ms over 2 steps
    r = b.make_roofline("rankb_tc", "f32_3xtf32", 2e9, 2e12, 20.0, 4, 2)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 100.0) < 1e-9
    want_peak = peaks["bf16_tflops_sustained"] * 1.1 / 2.25 / 3.0
    assert abs(r["peak"] - want_peak) < 1e-9 and abs(r["frac"] - 100.0 / want_peak) < 1e-12
    assert r["kernel_ms_per_step"] == 10.0 and r["kernel_launches_per_step"] == 2
    # any other kernel is reported against HBM: 6.6e9 bytes in 1 s
    r = b.make_roofline("panel", "f32_3xtf32", 6.6e9, 0.0, 1000.0, 1, 1)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 6.6) < 1e-9 and r["peak"] == peaks["hbm_gbs"]
    # BF16x3 and plain TF32 peaks
    assert abs(b.make_roofline("rankb_tc", "f32_bf16x3", 1, 1, 1, 1, 1)["peak"]
               - peaks["bf16_tflops_sustained"] / 3.0) < 1e-9
    assert abs(b.make_roofline("rankb_tc", "f32_tf32", 1, 1, 1, 1, 1)["peak"]
               - peaks["bf16_tflops_sustained"] * 1.1 / 2.25) < 1e-9


def test_sweep_roofline_arithmetic():
    """The sweep-level figure: 2N^3/3 useful flop over the step time, against the
    tensor peak of the mode's arithmetic; the panel chain as time per pivot."""
    b = _bench_module()
    N, ms = 32768, 200.0
    shares = {"panel": {"launches": 256, "ms": 120.0, "bytes": 0.0, "flops": 0.0, "share": 0.5},
              "rankb_tc": {"launches": 600, "ms": 120.0, "bytes": 1e12, "flops": 2e13,
                           "share": 0.5}}
    r = b.sweep_roofline("f32_3xtf32", N, ms, shares)
    want = 2.0 * N ** 3 / 3.0 / 0.2 / 1e12
    assert abs(r["achieved"] - want) < 1e-9
    assert r["bound"] == "tensor" and abs(r["frac"] - want / b.tensor_peak("f32_3xtf32")[0]) < 1e-12
    assert abs(r["pivot_chain"]["us_per_pivot"] - 120e3 / N) < 1e-12
    assert abs(r["tensor_update"]["achieved"] - 2e13 / 0.12 / 1e12) < 1e-9
    # a plain mode reports its rank-1 update against HBM
    r = b.sweep_roofline("f64_plain", 8000, 600.0, {
        "update": {"launches": 8000, "ms": 500.0, "bytes": 3e12, "flops": 1e11, "share": 0.9}})
    assert r["bound"] == "hbm" and abs(r["achieved"] - 3e12 / 0.5 / 1e9) < 1e-6
