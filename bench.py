"""Benchmark of the sparse MTTKRP / CP-ALS hot path on GB300.

One step = the whole path on one synthetic tensor already resident in HBM:
relate_encode (GPU key build, radix sort, partitions, statistics) followed by
relate_cpals for the workload's iteration count (MTTKRP of every mode, FP64
normal equations, normalisation, fit) from the same initial factors.

value = MTTKRP work of the step (nnz * R * N * iterations) / step time,
summed over ranks (replicas, weak scaling) and divided by the slowest rank's
time. e2e = the same through the C ABI with host buffers: pinned host
coordinates, values and factors copied in and the factors and lambda copied
out inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload NAME] [--factor-dtype f32|bf16|f64]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "zipf3d-200Kx200Kx5K-50M"
METRIC = "MTTKRP nnz*R/s (all modes, whole CP-ALS job)"
UNIT = "nnz*R/s"
CPU_SAMPLE_NNZ = 5_000_000  # nonzeros of the workload the CPU oracle runs per step

# DRAM traffic of the MTTKRP kernel per launch from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only while the kernel
# source is unchanged (sha256 of csrc/mttkrp_impl.cuh). None = not captured.
NCU_TRAFFIC = {"sha256": "b95f435e32cd5dd9716be6ae0ccdfb7600a6e49460af90a901e7ebb066b690b6",
               # 20M-nonzero capture (336.9 MB per launch), stream part (8-byte
               # word, 4-byte value, 2-byte tile-order entry) scaled to 50M
               # nonzeros: 336.9 MB + 30M x 14 B
               "bytes_per_launch": 756.9e6, "workload": "zipf3d-200Kx200Kx5K-50M"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_sha() -> str:
    """sha256 over the code of the MTTKRP kernel and its launch configuration
    (comments and blank lines removed, so that editing a comment does not
    invalidate the ncu counters)."""
    import re
    h = hashlib.sha256()
    for name in ("mttkrp_impl.cuh", "mttkrp.cu"):
        with open(os.path.join(ROOT, "paper_2509_00280_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        return dist, world, rank, local
    return None, 1, 0, local


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _load_workload(name: str):
    import synth
    w = synth.WORKLOADS[name]
    coords, vals = synth.make_tensor(w["spec"])
    return w, coords, vals


def _algorithmic_bytes(stats, mode, R, fb, ab, vb):
    """Compulsory HBM bytes of one mode-n MTTKRP: the stream (word + value),
    each distinct row of the other factors once, the output written once."""
    nnz = stats["nnz"]
    b = nnz * (stats["key_bytes"] + vb)
    for k in range(stats["nmodes"]):
        if k != mode:
            b += stats["distinct"][k] * R * fb
    b += stats["dims"][mode] * R * ab
    return b


def _launches_per_step(stats, iters, fdt, n_tile_orders, R):
    """Kernel launches of one step, counted from the library's launch
    sequence (and checked against an ncu launch list):
    encode = key build, 5 kernels per radix pass of the keys (ceil(l(p)/8)
    passes) and of each mode's hot-row count sort (4 passes), word packing,
    gather, partition statistics, per mode a histogram summary, a count and
    a hot-row list, and the 2-kernel norm;
    CP-ALS = the initial Grams (partial + reduce per mode), one tile order per
    SEGMENTED mode, and per iteration per mode: normal equations, MTTKRP,
    then row pass + Gram (fused) + reduce + finish + store (FP32/FP64) or row
    pass + 2 column-norm kernels + store + tensor-core Gram + reduce +
    inner products (BF16), plus the fit and the kernel that records it."""
    N = stats["nmodes"]
    passes = (stats["lp"] + 7) // 8
    encode = 1 + 5 * (passes + 4 * N) + 1 + 1 + 1 + 3 * N + 2
    per_mode = 9 if (fdt == "bf16" and R % 8 == 0) else 6
    # graph replay with a fixed iteration count records each fit (1 kernel)
    cpals = 2 * N + n_tile_orders + iters * (per_mode * N + 1 + 1)
    return encode + cpals


def run_cpu_reference(args, w, coords, vals, sample_nnz: int, iters: int = 1):
    """The oracle as it stands (single-threaded C, FP64) on a bounded sample
    of the same workload: CP-ALS iterations on the first sample_nnz nonzeros."""
    import oracle
    spec = w["spec"]
    R = w["R"]
    c = np.ascontiguousarray(coords[:, :sample_nnz])
    v = vals[:sample_nnz].astype(np.float64)
    fs = __import__("synth").init_factors(spec.dims, R, seed=0)
    t0 = time.perf_counter()
    oracle.cpals(c, v, spec.dims, R, iters, 0.0, fs)
    dt = time.perf_counter() - t0
    units = sample_nnz * R * len(spec.dims) * iters
    return (units / dt if iters else 0.0), dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--factor-dtype", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-kernel", action="store_true",
                    help="encode once and time only the per-mode MTTKRP launches (profiling runs)")
    args = ap.parse_args()

    dist, world, rank, local = _dist_setup()
    import torch
    import synth

    w = synth.WORKLOADS[args.workload]
    spec = w["spec"]
    R, iters = w["R"], w["iters"]
    fdt = args.factor_dtype or w["factor_dtype"]
    N = len(spec.dims)
    workload_cfg = {"workload": spec.name, "dims": list(spec.dims), "nnz": spec.nnz, "R": R, "iters": iters,
                    "factor_dtype": fdt, "acc_dtype": "f64" if fdt == "f64" else "f32",
                    "values": spec.values, "distributions": [list(d) for d in spec.dists]}

    if args.impl == "reference":
        if rank != 0:
            return
        _, coords, vals = _load_workload(args.workload)
        sample = min(spec.nnz, CPU_SAMPLE_NNZ)
        for _ in range(args.warmup):
            run_cpu_reference(args, w, coords, vals, min(sample, 10_000), iters=0)
        times, units = [], 0
        for _ in range(args.steps):
            thr, dt = run_cpu_reference(args, w, coords, vals, sample)
            times.append(dt)
            units += sample * R * N
        total = sum(times)
        val = units / total
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {**workload_cfg, "sample_nnz": sample, "iters_per_step": 1},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"first {sample} nonzeros of {spec.name}, 1 CP-ALS iteration "
                                           f"(all {N} modes) per step, single-threaded C oracle"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import paper_2509_00280_gb300 as rl
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    _, coords, vals = _load_workload(args.workload)
    t_gen = time.perf_counter() - t_gen
    torch_fdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[fdt]
    vals_in = vals.astype(np.float64) if fdt == "f64" else vals
    d_coords = torch.from_numpy(coords).to(dev)
    d_vals = torch.from_numpy(vals_in).to(dev)
    init = synth.init_factors(spec.dims, R, seed=0)
    d_init = [torch.from_numpy(f).to(dev).to(torch_fdt).contiguous() for f in init]
    d_fac = [t.clone() for t in d_init]
    # a dedicated stream: relate_cpals replays a captured CUDA graph per ALS
    # iteration, which needs a non-default stream
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    if args.only_kernel:
        h = rl.relate_encode(d_coords, d_vals, spec.dims, factor_dtype=fdt, stream=stream)
        accdt = torch.float64 if fdt == "f64" else torch.float32
        for n in range(N):
            out = torch.empty((spec.dims[n], R), dtype=accdt, device=dev)
            for _ in range(max(1, args.steps)):
                rl.relate_mttkrp(h, n, d_fac, R, out, stream)
        torch.cuda.synchronize()
        h.close()
        print(json.dumps({"only_kernel": spec.name, "modes": N, "launches_per_mode": max(1, args.steps)}))
        return

    def step():
        for a, b in zip(d_fac, d_init):
            a.copy_(b)
        h = rl.relate_encode(d_coords, d_vals, spec.dims, factor_dtype=fdt, stream=stream)
        rl.relate_set_cpals_graph(h, True)
        res = rl.relate_cpals(h, R, iters, 0.0, d_fac)
        stats = rl.relate_get_stats(h)
        h.close()
        return res, stats

    for _ in range(args.warmup):
        res, stats = step()
    torch.cuda.synchronize()
    _barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            res, stats = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    _barrier(dist)
    t_ms = ev0.elapsed_time(ev1)
    t_ms = _max_over_ranks(dist, t_ms)
    units_step = spec.nnz * R * N * iters
    value = units_step * args.steps * world / (t_ms / 1000.0)

    # --- dominant kernel: per-mode MTTKRP launches timed with events on the stream
    h = rl.relate_encode(d_coords, d_vals, spec.dims, factor_dtype=fdt, stream=stream)
    stats = rl.relate_get_stats(h)
    accdt = torch.float64 if fdt == "f64" else torch.float32
    fb = {"f64": 8, "f32": 4, "bf16": 2}[fdt]
    ab = 8 if fdt == "f64" else 4
    vb = 8 if fdt == "f64" else 4
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    per_mode = []
    reps = 5
    for n in range(N):
        out = torch.empty((spec.dims[n], R), dtype=accdt, device=dev)
        ms = []
        for r in range(reps + 1):
            flush.fill_(float(r))  # 256 MB write evicts L2 between launches
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rl.relate_mttkrp(h, n, d_fac, R, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ms.append(e0.elapsed_time(e1))
        alg = _algorithmic_bytes(stats, n, R, fb, ab, vb)
        per_mode.append({"mode": n, "ms": statistics.mean(ms), "alg_bytes": alg,
                         "strategy": rl.relate_get_conflict(h, n, R)})
    h.close()
    alg_total = sum(m["alg_bytes"] for m in per_mode)
    ms_total = sum(m["ms"] for m in per_mode)
    achieved = (alg_total / N) / (ms_total / N / 1000.0) / 1e9
    peak, peak_kind = _peaks()
    traffic = None
    if NCU_TRAFFIC["sha256"] == _kernel_sha() and NCU_TRAFFIC["workload"] == spec.name:
        traffic = NCU_TRAFFIC["bytes_per_launch"]

    # --- e2e through the C ABI with host buffers
    pin_c = torch.from_numpy(coords).pin_memory()
    pin_v = torch.from_numpy(vals_in).pin_memory()
    pin_f = [torch.from_numpy(f).to(torch_fdt).contiguous().pin_memory() for f in init]
    out_f = [torch.empty_like(f).pin_memory() for f in pin_f]

    def e2e_step():
        for a, b in zip(d_fac, pin_f):
            a.copy_(b, non_blocking=True)
        h2 = rl.relate_encode(pin_c.numpy(), pin_v.numpy(), spec.dims, factor_dtype=fdt, stream=stream)
        rl.relate_set_cpals_graph(h2, True)
        r2 = rl.relate_cpals(h2, R, iters, 0.0, d_fac)
        for a, b in zip(out_f, d_fac):
            a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        h2.close()
        return r2

    e2e_step()
    torch.cuda.synchronize()
    _barrier(dist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(dist, e0.elapsed_time(e1))
    e2e_val = units_step * e2e_steps * world / (e2e_ms / 1000.0)
    h2d = coords.nbytes + vals_in.nbytes + sum(f.numel() * f.element_size() for f in pin_f)
    d2h = sum(f.numel() * f.element_size() for f in out_f) + R * 8

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fdt == "f64" else "f32",
            "data": "synthetic",
            "config": {**workload_cfg, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "step": f"encode + {iters} CP-ALS iterations (tol 0), one CUDA graph per iteration",
                       "l2": "inputs larger than L2 (stream %d MB); L2 flushed between kernel timings"
                             % (spec.nnz * (stats['key_bytes'] + vb) // 2 ** 20),
                       "final_fit": res["fit"]},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": _launches_per_step(stats, iters, fdt, sum(1 for m in per_mode if m["strategy"] == 2),
                                               R) * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "k_mttkrp", "per_mode": per_mode},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = min(spec.nnz, CPU_SAMPLE_NNZ)
        thr, dt = run_cpu_reference(args, w, coords, vals, sample)
        line["cpu_baseline"] = {"value": thr, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {sample} nonzeros, 1 CP-ALS iteration (all {N} modes), "
                                          f"single-threaded C oracle, {dt:.1f} s"}
    if rank == 0:
        print(f"# generation {t_gen:.1f} s; per-mode MTTKRP ms {[round(m['ms'], 3) for m in per_mode]}",
              file=sys.stderr)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
