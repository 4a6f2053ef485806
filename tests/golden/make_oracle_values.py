"""Writes stored oracle results for large seeded inputs (calls only ``oracle/``).

The values are produced by the CPU oracle on inputs from ``workloads`` whose
generation is platform-independent (numpy's default_rng normal draws, no BLAS),
so the GPU side can regenerate the identical matrix anywhere.

    python tests/golden/make_oracle_values.py [--threads T]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

CASES = {
    # dense iid N(0, 1/N), N = 8000, seed 1 (the first matrix drawn from seed 1)
    "dense_n8000_seed1": lambda: workloads.dense_gaussian(8000, seed=1, var=1.0 / 8000),
    # dense iid N(0, 1), N = 1000, seed 0
    "dense_n1000_seed0": lambda: workloads.dense_gaussian(1000, seed=0),
    # SPD X^T X / (2N) + 1e-3 I, N = 8000, X drawn from seed 1 after the dense
    # matrix above (the product X^T X is a BLAS call: another host's BLAS may
    # round it differently, far below the 1e-12 tolerance of the FP64 paths)
    "spd_n8000_seed1": lambda: workloads.dense_and_spd_pair(8000, seed=1)[1],
}
GENERATORS = {"dense_n8000_seed1": "workloads.dense_gaussian",
              "dense_n1000_seed0": "workloads.dense_gaussian",
              "spd_n8000_seed1": "workloads.dense_and_spd_pair(...)[1]"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    for name, make in CASES.items():
        if args.only and name != args.only:
            continue
        A = make()
        t0 = time.time()
        res = oracle.logdet(A, nthreads=args.threads)
        dt = time.time() - t0
        out = {
            "case": name,
            "generator": GENERATORS[name],
            "n": int(A.shape[0]),
            "sign": res.sign,
            "logabs": res.logabs,
            "logabs_hex": float(res.logabs).hex(),
            "piv_label_sha": __import__("hashlib").sha256(res.piv_label.astype(np.int64).tobytes()).hexdigest(),
            "piv_value_sha": __import__("hashlib").sha256(res.piv_value.astype(np.float64).tobytes()).hexdigest(),
            "written_by": "tests/golden/make_oracle_values.py (oracle.logdet, FP64)",
            "oracle_seconds": round(dt, 2),
            "threads": args.threads,
        }
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, res.sign, res.logabs, f"{dt:.1f}s", flush=True)


if __name__ == "__main__":
    main()
