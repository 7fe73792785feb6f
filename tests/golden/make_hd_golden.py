"""Write the oracle's results on the 1920x1080 D=256 synthetic pair into hd_1920x1080_d256.json
(and its FP64-form disparities into hd_1920x1080_d256_f64_disp.npz).

The full-HD configuration: one seeded 1920x1080 pair (synth.WORKLOADS["hd_1920x1080_d256"]),
256 labels, 9x9 NCC window, data costs quantised with trunc 20, 4 scales, 10 iterations per
scale, lambda 10, trunc 2, the exact fast-converging skip.  Both forms of the method are run
through the CPU oracle only (section "Correlation volume computation" for the cost,
sections "Fast Converging BP" and "GPU Implementation" for the solve, section "Approach
Description" for the energy):

  int  -- the quantised integer method: SHA-256 of the int32 cost volume [H][W][D] and of the
          int32 disparities [H][W] (little-endian bytes), the int64 energy, the skip trace;
  f64  -- the FP64 reference of the float-message form (unquantised cost, FP64 messages):
          its FP64 energy on that cost (exact bits as float.hex), its trace, the SHA-256 of
          its disparities, and the disparities themselves (uint8, compressed), against which
          the fp16-message form's energy gap and label disagreement are measured.

Nothing here runs on a GPU or imports the CUDA package; the generator module holds no part
of the method.  The oracle's OpenMP build is used when it is available (same bits as the
serial build).  About 20 minutes on 8 cores and 40 GB of host memory.

    python tests/golden/make_hd_golden.py [--threads N]
"""
from __future__ import annotations

import argparse
import base64
import hashlib
import json
import os
import platform
import sys
import time
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1709_06509_gb300 import synth  # noqa: E402

NAME = "hd_1920x1080_d256"
TRUNC_DATA, LEVELS, ITERS, LAM, TRUNC = 20, 4, 10, 10, 2
LATTICE = 8


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def lattice(disp: np.ndarray) -> str:
    """Every LATTICE-th label of every LATTICE-th row, uint8, zlib, base64: for locating a mismatch."""
    return base64.b64encode(zlib.compress(disp[::LATTICE, ::LATTICE].astype(np.uint8).tobytes(), 9)).decode()


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    pair, window = synth.workload_pair(NAME)
    H, W = pair.left.shape
    D = pair.D
    use_omp = oracle.openmp_available()
    ctx = oracle.openmp(args.threads) if use_omp else None
    threads = ctx.__enter__() if ctx else 1
    t0 = time.perf_counter()
    ncc = oracle.ncc(pair.left, pair.right, D, window)
    cost_i = oracle.quantise(ncc, TRUNC_DATA)
    cost_f = oracle.cost_float(ncc, TRUNC_DATA)
    del ncc
    t1 = time.perf_counter()
    disp_i, trace_i = oracle.bp_wta(cost_i, LEVELS, ITERS, LAM, TRUNC, skip=True)
    t2 = time.perf_counter()
    energy_i = oracle.energy(cost_i, disp_i, LAM, TRUNC)
    cost_sha = sha(cost_i.astype("<i4"))
    del cost_i
    t3 = time.perf_counter()
    disp_f, trace_f = oracle.bp_wta(cost_f, LEVELS, ITERS, float(LAM), TRUNC, skip=True)
    t4 = time.perf_counter()
    energy_f = oracle.energy(cost_f, disp_f, float(LAM), TRUNC)
    if ctx:
        ctx.__exit__(None, None, None)
    out = {
        "workload": NAME, "W": W, "H": H, "D": D, "window": window, "trunc_data": TRUNC_DATA, "levels": LEVELS,
        "iters": ITERS, "lambda": LAM, "trunc": TRUNC, "fast_skip": True,
        "left_sha256": sha(pair.left), "right_sha256": sha(pair.right),
        "int": {"cost_sha256": cost_sha, "disp_sha256": sha(disp_i.astype("<i4")), "energy": int(energy_i),
                "trace": [int(v) for v in trace_i], "disp_lattice": lattice(disp_i)},
        "f64": {"energy_hex": float(energy_f).hex(), "energy": float(energy_f),
                "disp_sha256": sha(disp_f.astype("<i4")), "trace": [int(v) for v in trace_f],
                "disp_lattice": lattice(disp_f), "disp_file": NAME + "_f64_disp.npz"},
        "lattice_step": LATTICE,
        "oracle_run": {"threads": threads, "openmp": use_omp, "machine": platform.machine(),
                       "seconds": {"ncc_and_costs": round(t1 - t0, 1), "int_bp_wta": round(t2 - t1, 1),
                                   "f64_bp_wta": round(t4 - t3, 1)}},
    }
    np.savez_compressed(os.path.join(HERE, NAME + "_f64_disp.npz"), disp=disp_f.astype(np.uint8))
    with open(os.path.join(HERE, NAME + ".json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out["oracle_run"]))


if __name__ == "__main__":
    main()
