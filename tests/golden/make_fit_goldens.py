"""Writes tests/golden/fit_<workload>.txt: the FP64 CP-ALS fit trace of the CPU
oracle on a full-size workload, for the GPU tests that compare the library's
FP64 / FP32 / BF16 CP-ALS with it.

Calls only the oracle (oracle.cpals: plain single-threaded FP64 CP-ALS) and
the seeded input generator (synth); nothing of the CUDA path. Inputs: the
workload's tensor (values rounded to their stored dtype, then taken exactly
in FP64) and synth.init_factors(dims, R, seed=0) in FP64. The SHA-256 of the
coordinate and value arrays is recorded so that a test can check that the
box regenerates the same tensor.

Usage: python tests/golden/make_fit_goldens.py WORKLOAD [ITERS]
(the full-size workloads take minutes to about an hour of one core each).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def tensor_sha256(coords: np.ndarray, vals: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(coords).tobytes())
    h.update(np.ascontiguousarray(vals).tobytes())
    return h.hexdigest()


def main() -> None:
    name = sys.argv[1]
    w = synth.WORKLOADS[name]
    spec = w["spec"]
    iters = int(sys.argv[2]) if len(sys.argv) > 2 else w["iters"]
    R = w["R"]
    coords, vals = synth.make_tensor(spec)
    sha = tensor_sha256(coords, vals)
    fs = synth.init_factors(spec.dims, R, seed=0)
    t0 = time.time()
    res = oracle.cpals(coords, vals.astype(np.float64), spec.dims, R, iters, 0.0, fs)
    dt = time.time() - t0
    out = os.path.join(ROOT, "tests", "golden", f"fit_{name}.txt")
    with open(out, "w") as f:
        f.write(f"# FP64 CP-ALS fit trace of the CPU oracle (oracle.cpals) on {name}\n")
        f.write(f"# R = {R}, {iters} iterations, tol 0, initial factors synth.init_factors(dims, R, seed=0) in FP64\n")
        f.write("# fit = 1 - ||X - Xhat|| / ||X|| after each iteration (Gauss-Seidel ALS, Cholesky with ridge retry)\n")
        f.write(f"# written by tests/golden/make_fit_goldens.py in {dt:.0f} s\n")
        f.write(f"tensor_sha256 {sha}\n")
        f.write(f"R {R}\n")
        f.write(f"iters {res['iters']}\n")
        f.write(f"ridges {res['ridges']}\n")
        f.write("fit_trace " + " ".join(f"{x:.17g}" for x in res["fit_trace"]) + "\n")
        f.write("lambda " + " ".join(f"{x:.17g}" for x in res["lam"]) + "\n")
    print(out, dt)


if __name__ == "__main__":
    main()
