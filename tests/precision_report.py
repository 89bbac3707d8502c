"""Measured error of every workload and factor precision against the FP64
oracle, written as a markdown table (profiles/precision_errors.md).

Run on a GPU machine from the repository root:
    python tests/precision_report.py > profiles/precision_errors.md

Per (workload, factor dtype):
* MTTKRP: the relative Frobenius error of the full-size launch (benchmark
  configuration, AUTO plan) on each mode's most populated and random rows,
  against the oracle's MTTKRP over exactly those rows' nonzeros (the method of
  tests/test_gpu_fullsize.py); the largest over the modes is reported. BF16 is
  reported against the oracle fed the BF16-rounded factors (the arithmetic's
  error) and against the unrounded factors (the acceptance number).
* CP-ALS: the final fit of the library's CP-ALS (graph replay, tol 0, the
  workload's iteration count) and its distance to the oracle's FP64 fit
  (tests/golden/fit_<workload>.txt).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import synth  # noqa: E402
import paper_2509_00280_gb300 as rl  # noqa: E402
from conftest import read_golden  # noqa: E402
from gpu_util import factors_dev, rel_fro  # noqa: E402
from test_gpu_fit_golden import run_cpals  # noqa: E402
from test_gpu_fullsize import _mttkrp_rows, _oracle_rows, _sample_rows  # noqa: E402

CASES = [("uniform3d-1000x1000x1000-1M", "f64"),
         ("zipf3d-200Kx200Kx5K-50M", "f32"), ("zipf3d-200Kx200Kx5K-50M", "bf16"),
         ("zipf4d-5Mx1Mx100Kx24-150M", "f64"), ("zipf4d-5Mx1Mx100Kx24-150M", "f32"),
         ("zipf4d-5Mx1Mx100Kx24-150M", "bf16"),
         ("zipf5d-10Mx10Mx1Mx1Kx100-100M", "bf16"), ("zipf5d-10Mx10Mx1Mx1Kx100-100M", "f64")]
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 2e-2}


def mttkrp_errors(name, fdt):
    w = synth.WORKLOADS[name]
    spec, R = w["spec"], w["R"]
    c, v = synth.make_tensor(spec)
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float64 if fdt == "f64" else np.float32)
    fs_unr = [f.astype(np.float64) for f in fs]
    fs_rnd = [oracle.round_bf16(f).astype(np.float64) for f in fs] if fdt == "bf16" else fs_unr
    dfs = factors_dev(fs, fdt)
    v64 = v.astype(np.float64)
    h = rl.relate_encode(torch.from_numpy(c).cuda(), torch.from_numpy(v).cuda(), spec.dims, factor_dtype=fdt)
    rng = np.random.default_rng(7)
    err_rnd, err_unr = 0.0, 0.0
    for n in range(len(spec.dims)):
        rows = _sample_rows(np.bincount(c[n], minlength=spec.dims[n]), rng)
        if rows.size == 0:
            continue
        got = _mttkrp_rows(h, n, dfs, R, rows, fdt=fdt)
        err_rnd = max(err_rnd, rel_fro(got, _oracle_rows(c, v64, spec.dims, n, rows, fs_rnd)))
        if fdt == "bf16":
            err_unr = max(err_unr, rel_fro(got, _oracle_rows(c, v64, spec.dims, n, rows, fs_unr)))
    h.close()
    return err_rnd, err_unr


def main():
    print("# Measured error against the FP64 oracle, per workload and factor precision")
    print()
    print("Command (GB300, from the repository root): `python tests/precision_report.py > "
          "profiles/precision_errors.md`.")
    print("MTTKRP: largest relative Frobenius error over the modes, full-size launch, sampled rows (each "
          "mode's 8 most populated rows within 4M nonzeros plus 56 random populated rows) against the oracle "
          "over exactly those rows' nonzeros; BF16 against the rounded factors and (acceptance) the unrounded "
          "ones. CP-ALS: final fit after the workload's iterations (tol 0, graph replay) and its distance to "
          "the oracle's FP64 fit (tests/golden/fit_*.txt).")
    print()
    print("| workload | factors | MTTKRP error | bound | CP-ALS fit | oracle FP64 fit | abs(fit - FP64 fit) | bound |")
    print("|---|---|---|---|---|---|---|---|")
    for name, fdt in CASES:
        t0 = time.time()
        e_rnd, e_unr = mttkrp_errors(name, fdt)
        g = read_golden(f"fit_{name}.txt")
        gold = np.array([float(x) for x in g["fit_trace"]])
        res, _ = run_cpals(name, fdt, len(gold))
        mt = f"{e_rnd:.2e}" if fdt != "bf16" else f"{e_rnd:.2e} (rounded) / {e_unr:.2e} (unrounded)"
        fit_bound = "1e-9 (every iteration)" if fdt == "f64" else "1e-3"
        dfit = float(np.max(np.abs(res["fit_trace"] - gold))) if fdt == "f64" else abs(res["fit"] - gold[-1])
        print(f"| {name} | {fdt} | {mt} | {TOL[fdt]:.0e} | {res['fit']:.10f} | {gold[-1]:.10f} | {dfit:.2e} | "
              f"{fit_bound} |", flush=True)
        print(f"# {name} {fdt}: {time.time() - t0:.0f} s", file=sys.stderr, flush=True)


if __name__ == "__main__":
    main()
