"""Benchmark of the sparse MTTKRP / CP-ALS hot path on GB300.

One step = the whole path on one synthetic tensor already resident in HBM:
relate_encode (GPU key build, radix sort, partitions, statistics) followed by
relate_cpals for the workload's iteration count (MTTKRP of every mode, FP64
normal equations, normalisation, fit) from the same initial factors.

Default: the 4-mode 150M-nonzero workload (5M x 1M x 100K x 24, R = 64, 10
iterations) with FP64 factors and accumulation, the paper's precision
(Sec. 4.1.3); the FP32 and BF16 factor forms of the same workload are timed
after it and reported under "variants".

value = MTTKRP work of the step (nnz * R * N * iterations) / step time,
summed over ranks (replicas, weak scaling) and divided by the slowest rank's
time. e2e = the same through the C ABI with host buffers: pinned host
coordinates, values and factors copied in and the factors and lambda copied
out inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--workload NAME] [--factor-dtype f64|f32|bf16] [--variants f32,bf16]
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

DEFAULT_WORKLOAD = "zipf4d-5Mx1Mx100Kx24-150M"
DEFAULT_FACTOR_DTYPE = "f64"  # the paper's precision (Sec. 4.1.3)
DEFAULT_VARIANTS = "f32,bf16"
METRIC = "MTTKRP nnz*R/s (all modes, whole CP-ALS job)"
UNIT = "nnz*R/s"
CPU_SAMPLE_NNZ = 30_000_000    # nonzeros of the workload the OpenMP CPU baseline sweeps
CPU_SINGLE_NNZ = 1_000_000     # nonzeros the single-threaded oracle sweeps (reported beside it)
REF_SAMPLE_NNZ = 10_000_000    # nonzeros per step of the --impl reference arm
# FP64 issue rate of a GB300 SM: 2 FP64 FMA per clock (a register-only FMA
# loop measures 626 G FMA/s on 152 SMs at 2070 MHz, 1.99 per SM per clock)
FP64_FMA_PER_SM_CLK = 2
NUM_SMS = 152

# DRAM traffic of the MTTKRP kernel per launch from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only while the kernel
# source is unchanged (sha256 of csrc/mttkrp_impl.cuh). None = not captured.
NCU_TRAFFIC = {"sha256": "d0051ef187efbb77cb10433766bc0705194893553b17aade8d9238a0092e3e3e",
               # full-size 1-pass capture (dram__bytes_read.sum + dram__bytes_write.sum)
               # of the 4 per-mode launches of the FP64 factored MTTKRP (modes 0-2 with
               # their Khatri-Rao pairs), their mean
               "bytes_per_launch": 28.66e9, "workload": "zipf4d-5Mx1Mx100Kx24-150M", "dtype": "f64"}


# L1 / L2 traffic of the MTTKRP kernels from ncu captures of smaller cases of
# the same workload families (l1tex__t_bytes.sum and lts__t_bytes.sum, mean
# per launch over the modes), scaled to a launch of the timed workload by its
# nonzero count: the cache traffic of a launch is proportional to its
# nonzeros (the FP64 case captured with the Khatri-Rao pairs of modes 0-2 on,
# as the AUTO plans of the 150M-nonzero case). Filled from
# profiles/k_mttkrp_cache_traffic.md.
_SHA_CACHE = "d0051ef187efbb77cb10433766bc0705194893553b17aade8d9238a0092e3e3e"
NCU_CACHE = [
    {"sha256": _SHA_CACHE, "family": "zipf4d-5Mx1Mx100Kx24", "dtype": "f64", "workload": "zipf4d-5Mx1Mx100Kx24-30M",
     "nnz": 30e6, "l1_bytes": 3.472e10, "l2_bytes": 3.717e10},
    {"sha256": _SHA_CACHE, "family": "zipf4d-5Mx1Mx100Kx24", "dtype": "f32", "workload": "zipf4d-5Mx1Mx100Kx24-30M",
     "nnz": 30e6, "l1_bytes": 2.413e10, "l2_bytes": 1.425e10},
    {"sha256": _SHA_CACHE, "family": "zipf4d-5Mx1Mx100Kx24", "dtype": "bf16", "workload": "zipf4d-5Mx1Mx100Kx24-30M",
     "nnz": 30e6, "l1_bytes": 1.280e10, "l2_bytes": 7.759e9},
    {"sha256": _SHA_CACHE, "family": "zipf3d-200Kx200Kx5K", "dtype": "f32", "workload": "zipf3d-200Kx200Kx5K-20M",
     "nnz": 20e6, "l1_bytes": 5.255e9, "l2_bytes": 2.007e9},
]


def _cache_rates(fdt, workload, nnz, sec_per_launch):
    family = workload.rsplit("-", 1)[0]
    for c in NCU_CACHE:
        if c["sha256"] == _kernel_sha() and c["family"] == family and c["dtype"] == fdt:
            scale = nnz / c["nnz"]
            return {"l1_gbs": c["l1_bytes"] * scale / sec_per_launch / 1e9,
                    "l2_gbs": c["l2_bytes"] * scale / sec_per_launch / 1e9,
                    "source": f"ncu l1tex__t_bytes.sum / lts__t_bytes.sum of {c['workload']}, scaled to {int(nnz)} nonzeros"}
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _fp64_peak_tflops():
    """FP64 arithmetic peak from unit counts and the clock: 152 SMs x 2 FMA
    (4 flops) per SM per clock x the maximum SM clock (MEASURED_PEAKS.json's
    sm_max_mhz, else 2070 MHz) = 1.26 TFLOP/s, the nominal 1.25."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return NUM_SMS * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12


def _kernel_sha() -> str:
    """sha256 over the code of the MTTKRP kernel and its launch configuration
    (comments and blank lines removed, so that editing a comment does not
    invalidate the ncu counters)."""
    import re
    h = hashlib.sha256()
    for name in ("mttkrp_impl.cuh", "mttkrp.cu", "mttkrp_fac.cuh"):
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


def _kr_builds(kr_pairs):
    """Khatri-Rao tables built per CP-ALS iteration: mode n's MTTKRP builds
    its pair's table unless the last one built holds the same two modes and
    neither was updated since (each iteration starts with none)."""
    built, held = 0, None
    for n, pair in enumerate(kr_pairs or []):
        if pair is not None and tuple(pair) != held:
            built, held = built + 1, tuple(pair)
        if held is not None and n in held:
            held = None  # A_n is rewritten after its MTTKRP
    return built


def _launches_per_step(stats, iters, fdt, n_tile_orders, R, kr_pairs=None):
    """Kernel launches of one step, counted from the library's launch
    sequence (and checked against an ncu launch list):
    encode = key build, 5 kernels per radix pass of the keys (ceil(l(p)/8)
    passes) and of each mode's hot-row count sort (4 passes), word packing,
    gather, partition statistics, per mode a histogram summary, a count and
    a hot-row list, and the 2-kernel norm;
    CP-ALS = the initial Grams, one tile order per SEGMENTED mode, and per
    iteration per mode: normal equations, MTTKRP, then
      FP64: tensor-core row pass, column exponents + tensor-core Gram +
            reduce, finish, store (the initial Grams: exponents, Gram, reduce);
            a mode with I R (3R + 1) / 2 <= 8e6 FMA runs its row pass and
            Gram (partials + reduce) on the FP64 pipe instead, one kernel
            fewer per update and per initial Gram;
      FP32 rows (FP32 factors, or BF16 with R % 8 != 0): row pass,
            tensor-core Gram + reduce, finish, store;
      BF16: row pass, 2 column-norm kernels, store, tensor-core Gram of the
            stored factor + reduce, inner products;
    plus the fit and the kernel that records it, and per iteration the
    Khatri-Rao table builds of fused modes (_kr_builds)."""
    N = stats["nmodes"]
    passes = (stats["lp"] + 7) // 8
    encode = 1 + 5 * (passes + 4 * N) + 1 + 1 + 1 + 3 * N + 2
    if fdt == "f64":
        dims = stats.get("dims") or [1 << 62] * N
        small = sum(1 for I in dims if I * R * (3 * R + 1) / 2 <= 8e6)
        per_mode, init = 8 * N - small, 3 * N - small
    elif fdt == "bf16" and R % 8 == 0:
        per_mode, init = 9 * N, 2 * N
    else:
        per_mode, init = 7 * N, 2 * N
    # graph replay with a fixed iteration count records each fit (1 kernel)
    cpals = init + n_tile_orders + iters * (per_mode + 1 + 1 + _kr_builds(kr_pairs))
    return encode + cpals


def _host_cores():
    """Threads the CPU legs use: the cores this process may run on."""
    try:
        aff = sorted(os.sched_getaffinity(0))
    except Exception:
        aff = list(range(os.cpu_count() or 1))
    return len(aff), aff


def _affinity_str(aff) -> str:
    if not aff:
        return ""
    runs, a = [], aff[0]
    prev = a
    for x in aff[1:] + [None]:
        if x is not None and x == prev + 1:
            prev = x
            continue
        runs.append(f"{a}-{prev}" if prev != a else f"{a}")
        if x is not None:
            a = prev = x
    return ",".join(runs)


def _cpu_sweep(coords, vals, dims, factors, nthreads, sweeps):
    """Median time of `sweeps` all-mode MTTKRP sweeps of the oracle's OpenMP
    build (oracle_omp.c) on nthreads threads."""
    import oracle
    outs = [np.empty((int(d), factors[0].shape[1]), dtype=np.float64) for d in dims]
    oracle.mttkrp_omp(coords[:, :1000], vals[:1000], dims, 0, factors, nthreads, out=outs[0])  # load, warm
    times = []
    for _ in range(sweeps):
        t0 = time.perf_counter()
        for n in range(len(dims)):
            oracle.mttkrp_omp(coords, vals, dims, n, factors, nthreads, out=outs[n])
        times.append(time.perf_counter() - t0)
    return statistics.median(times)


def cpu_baseline(w, coords, vals):
    """The oracle's MTTKRP on the host cores: the OpenMP build on every core
    this process may use (all-mode sweeps, median of 3, on the first
    CPU_SAMPLE_NNZ nonzeros), and the plain single-threaded compensated
    oracle (one all-mode sweep on the first CPU_SINGLE_NNZ nonzeros)."""
    import oracle
    import synth
    spec, R = w["spec"], w["R"]
    N = len(spec.dims)
    fs = synth.init_factors(spec.dims, R, seed=0)
    cores, aff = _host_cores()
    n_omp = min(spec.nnz, CPU_SAMPLE_NNZ)
    c = np.ascontiguousarray(coords[:, :n_omp])
    v = vals[:n_omp].astype(np.float64)
    dt = _cpu_sweep(c, v, spec.dims, fs, cores, 3)
    omp_val = n_omp * R * N / dt
    n1 = min(spec.nnz, CPU_SINGLE_NNZ)
    c1 = np.ascontiguousarray(coords[:, :n1])
    v1 = vals[:n1].astype(np.float64)
    t0 = time.perf_counter()
    for n in range(N):
        oracle.mttkrp(c1, v1, spec.dims, n, fs)
    dt1 = time.perf_counter() - t0
    return {"value": omp_val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_omp} nonzeros of {spec.name} (R = {R}), all {N} modes per sweep, median of 3 "
                      f"sweeps ({dt:.2f} s each): OpenMP build of the oracle MTTKRP (oracle_omp.c, FP64) on "
                      f"{cores} threads",
            "nproc": os.cpu_count(), "affinity": _affinity_str(aff),
            "single_thread": {"value": n1 * R * N / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {n1} nonzeros, one all-mode sweep of the compensated "
                                        f"single-threaded oracle (oracle.c), {dt1:.2f} s"}}


def run_reference(args, w, coords, vals, world):
    """--impl reference: the oracle's MTTKRP (OpenMP build, FP64, every core
    this process may use) on a bounded sample of the same workload; a step is
    one all-mode MTTKRP sweep over the first REF_SAMPLE_NNZ nonzeros."""
    import synth
    spec, R = w["spec"], w["R"]
    N = len(spec.dims)
    cores, aff = _host_cores()
    n = min(spec.nnz, REF_SAMPLE_NNZ)
    c = np.ascontiguousarray(coords[:, :n])
    v = vals[:n].astype(np.float64)
    fs = synth.init_factors(spec.dims, R, seed=0)
    for _ in range(args.warmup):
        _cpu_sweep(c[:, :100_000], v[:100_000], spec.dims, fs, cores, 1)
    times = []
    for _ in range(args.steps):
        times.append(_cpu_sweep(c, v, spec.dims, fs, cores, 1))
    total = sum(times)
    val = n * R * N * args.steps / total
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": spec.name, "dims": list(spec.dims), "nnz": spec.nnz, "R": R,
                                            "sample_nnz": n, "step": "one all-mode MTTKRP sweep of the sample"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} nonzeros of {spec.name}, one all-mode MTTKRP sweep per step, "
                                       f"OpenMP build of the oracle (oracle_omp.c, FP64) on {cores} threads",
                             "nproc": os.cpu_count(), "affinity": _affinity_str(aff)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _time_kernels(rl, torch, h, stream, d_fac, spec, R, fdt, dev, reps):
    """Per-mode MTTKRP launch times (CUDA events on the launching stream, L2
    flushed by a 256 MB write before each launch) with their algorithmic
    bytes and flops."""
    N = len(spec.dims)
    stats = rl.relate_get_stats(h)
    accdt = torch.float64 if fdt == "f64" else torch.float32
    fb = {"f64": 8, "f32": 4, "bf16": 2}[fdt]
    ab = 8 if fdt == "f64" else 4
    vb = 8 if fdt == "f64" else 4
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    per_mode = []
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
        plan, kr = rl.relate_get_mode_plan(h, n, R), rl.relate_get_mode_kr(h, n, R)
        d = plan["depth"]
        per_mode.append({"mode": n, "ms": statistics.mean(ms), "alg_bytes": _algorithmic_bytes(stats, n, R, fb, ab, vb),
                         "alg_flops": spec.nnz * R * N, "strategy": rl.relate_get_conflict(h, n, R),
                         "kr_pair": plan["level"][d - 1:d + 1] if kr["kr"] else None})
    return stats, per_mode


def _roofline(per_mode, fdt, workload, nnz=None):
    """Roofline of the MTTKRP kernel over all modes: FP64 factors are bound by
    the FP64 pipe (flops = nnz * R * N per launch against the FP64 peak), FP32
    and BF16 factors against the measured HBM copy bandwidth (algorithmic
    bytes per launch)."""
    N = len(per_mode)
    ms_total = sum(m["ms"] for m in per_mode)
    peak_hbm, kind = _peaks()
    gbs = sum(m["alg_bytes"] for m in per_mode) / (ms_total / 1000.0) / 1e9
    hbm = {"achieved": gbs, "peak": peak_hbm, "unit": "GB/s", "frac": gbs / peak_hbm, "peak_kind": kind}
    traffic = None
    if NCU_TRAFFIC["sha256"] == _kernel_sha() and NCU_TRAFFIC["workload"] == workload and \
            NCU_TRAFFIC.get("dtype", "f32") == fdt:
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    cache = _cache_rates(fdt, workload, nnz, ms_total / 1000.0 / N) if nnz else None
    if fdt == "f64":
        tf = sum(m["alg_flops"] for m in per_mode) / (ms_total / 1000.0) / 1e12
        peak = _fp64_peak_tflops()
        return {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "traffic": traffic, "peak_kind": "derived: 152 SMs x 2 FP64 FMA per clock x 2 flops x max SM clock",
                "kernel": "k_mttkrp_fac", "hbm": hbm, "cache": cache, "per_mode": per_mode}
    return {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s", "frac": gbs / peak_hbm,
            "traffic": traffic, "peak_kind": kind, "kernel": "k_mttkrp", "cache": cache, "per_mode": per_mode}


def _time_dense(rl, torch, dev, I, R, fdt, reps):
    """CUDA-event time of relate_solve_rows and relate_gram on a random I x R
    matrix (each call includes its status read, one host sync)."""
    tdt = {"f64": torch.float64, "f32": torch.float32}[fdt if fdt in ("f64", "f32") else "f32"]
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    M = torch.rand((I, R), generator=g, device=dev, dtype=torch.float64).to(tdt)
    W = torch.rand((R, R), generator=g, device=dev, dtype=torch.float64) / R
    G = torch.empty((R, R), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    dt = "f64" if tdt == torch.float64 else "f32"
    out = {"only_dense": I, "R": R, "dtype": dt}
    for name, fn in (("solve_rows_ms", lambda: rl.relate_solve_rows(M, R, dt, W, st)),
                     ("gram_ms", lambda: rl.relate_gram(M, R, dt, G, st))):
        fn()
        t = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        out[name] = round(min(t), 3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--factor-dtype", default=None)
    ap.add_argument("--variants", default=None,
                    help="comma-separated factor dtypes timed after the main one (default f32,bf16 on the "
                         "default workload; 'none' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sharded", action="store_true",
                    help="with N > 1 GPUs: one tensor sharded over the ranks (contiguous equal-nnz slices of the "
                         "sorted stream, one NCCL all-reduce of M_n per mode; strong scaling) instead of replicas")
    ap.add_argument("--only-kernel", action="store_true",
                    help="encode once and time only the per-mode MTTKRP launches (profiling runs)")
    ap.add_argument("--plan-depth", type=int, default=None,
                    help="with --only-kernel: fiber-factoring depth of every mode (relate_set_mode_plan)")
    ap.add_argument("--plan-kr", type=int, default=-1, choices=(-1, 0, 1),
                    help="with --only-kernel: Khatri-Rao pair of every mode (relate_set_mode_kr; -1 AUTO)")
    ap.add_argument("--col-passes", type=int, default=0,
                    help="with --only-kernel: column passes of every mode (relate_set_mode_plan)")
    ap.add_argument("--only-dense", action="store_true",
                    help="time only the dense row update and Gram (relate_solve_rows, relate_gram) on a random "
                         "I x R matrix, I = the workload's longest mode (profiling runs)")
    ap.add_argument("--dense-rows", type=int, default=0, help="with --only-dense: I instead of the longest mode")
    args = ap.parse_args()

    dist, world, rank, local = _dist_setup()
    import synth

    w = synth.WORKLOADS[args.workload]
    spec = w["spec"]
    R, iters = w["R"], w["iters"]
    default_wl = args.workload == DEFAULT_WORKLOAD
    fdt = args.factor_dtype or (DEFAULT_FACTOR_DTYPE if default_wl else w["factor_dtype"])
    vlist = args.variants if args.variants is not None else (DEFAULT_VARIANTS if default_wl else "none")
    variants = [x for x in vlist.split(",") if x and x != "none" and x != fdt]
    if args.sharded and world > 1:
        variants = []  # the sharded line times the main precision only
    N = len(spec.dims)

    def wcfg(dt):
        return {"workload": spec.name, "dims": list(spec.dims), "nnz": spec.nnz, "R": R, "iters": iters,
                "factor_dtype": dt, "acc_dtype": "f64" if dt == "f64" else "f32",
                "values": spec.values, "distributions": [list(d) for d in spec.dists]}

    if args.impl == "reference":
        if rank != 0:
            return
        _, coords, vals = _load_workload(args.workload)
        print(json.dumps(run_reference(args, w, coords, vals, world)), flush=True)
        return

    import torch
    import paper_2509_00280_gb300 as rl
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only_dense:
        print(json.dumps(_time_dense(rl, torch, dev, args.dense_rows or max(spec.dims), R, fdt, max(1, args.steps))))
        return
    t_gen = time.perf_counter()
    _, coords, vals = _load_workload(args.workload)
    t_gen = time.perf_counter() - t_gen
    TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    init = synth.init_factors(spec.dims, R, seed=0)
    # a dedicated stream: relate_cpals replays a captured CUDA graph per ALS
    # iteration, which needs a non-default stream
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    def inputs(dt):
        # the values keep their stored dtype (FP32 values are exact in the FP64
        # arithmetic of FP64 factors)
        v_in = vals
        d_init = [torch.from_numpy(f).to(dev).to(TORCH_DT[dt]).contiguous() for f in init]
        return v_in, torch.from_numpy(coords).to(dev), torch.from_numpy(v_in).to(dev), d_init, \
            [t.clone() for t in d_init]

    vals_in, d_coords, d_vals, d_init, d_fac = inputs(fdt)

    if args.only_kernel:
        h = rl.relate_encode(d_coords, d_vals, spec.dims, factor_dtype=fdt, stream=stream)
        if args.plan_depth is not None or args.col_passes:
            for n in range(N):
                rl.relate_set_mode_plan(h, n, -1 if args.plan_depth is None else args.plan_depth, None,
                                        args.col_passes)
        for n in range(N):
            rl.relate_set_mode_kr(h, n, args.plan_kr)
        accdt = torch.float64 if fdt == "f64" else torch.float32
        ms = []
        for n in range(N):
            out = torch.empty((spec.dims[n], R), dtype=accdt, device=dev)
            t = []
            for _ in range(max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rl.relate_mttkrp(h, n, d_fac, R, out, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                t.append(e0.elapsed_time(e1))
            ms.append(round(min(t), 3))
        plans = [dict(rl.relate_get_mode_plan(h, n, R), kr=rl.relate_get_mode_kr(h, n, R)) for n in range(N)]
        h.close()
        print(json.dumps({"only_kernel": spec.name, "modes": N, "launches_per_mode": max(1, args.steps),
                          "factor_dtype": fdt, "ms_per_mode_min": ms, "plans": plans}))
        return

    sharded = args.sharded and world > 1

    def make_step(dt, dc, dv, dfac, dinit):
        def step():
            for a, b in zip(dfac, dinit):
                a.copy_(b)
            if sharded:  # this rank's slice of the sorted stream; M_n summed over the ranks
                from paper_2509_00280_gb300 import shard
                h = shard.sharded_encode(dc, dv, spec.dims, rank, world, factor_dtype=dt, stream=stream)
                res = shard.sharded_cpals(h, R, iters, 0.0, dfac)
            else:
                h = rl.relate_encode(dc, dv, spec.dims, factor_dtype=dt, stream=stream)
                rl.relate_set_cpals_graph(h, True)
                res = rl.relate_cpals(h, R, iters, 0.0, dfac)
            stats = rl.relate_get_stats(h)
            h.close()
            return res, stats
        return step

    step = make_step(fdt, d_coords, d_vals, d_fac, d_init)
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
    # replicas: every rank does the whole job (weak scaling); sharded: the
    # ranks share one job (strong scaling)
    value = units_step * args.steps * (1 if sharded else world) / (t_ms / 1000.0)

    # --- dominant kernel: per-mode MTTKRP launches timed with events on the stream
    h = rl.relate_encode(d_coords, d_vals, spec.dims, factor_dtype=fdt, stream=stream)
    stats, per_mode = _time_kernels(rl, torch, h, stream, d_fac, spec, R, fdt, dev, 5)
    h.close()
    roof = _roofline(per_mode, fdt, spec.name, spec.nnz)

    # --- e2e through the C ABI with host buffers
    pin_c = torch.from_numpy(coords).pin_memory()
    pin_v = torch.from_numpy(vals_in).pin_memory()
    pin_f = [torch.from_numpy(f).to(TORCH_DT[fdt]).contiguous().pin_memory() for f in init]
    out_f = [torch.empty_like(f).pin_memory() for f in pin_f]

    def e2e_step():
        for a, b in zip(d_fac, pin_f):
            a.copy_(b, non_blocking=True)
        if sharded:
            from paper_2509_00280_gb300 import shard
            h2 = shard.sharded_encode(pin_c.numpy(), pin_v.numpy(), spec.dims, rank, world, factor_dtype=fdt,
                                      stream=stream)
            r2 = shard.sharded_cpals(h2, R, iters, 0.0, d_fac)
        else:
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
    e2e_val = units_step * e2e_steps * (1 if sharded else world) / (e2e_ms / 1000.0)
    h2d = coords.nbytes + vals_in.nbytes + sum(f.numel() * f.element_size() for f in pin_f)
    d2h = sum(f.numel() * f.element_size() for f in out_f) + R * 8
    del pin_c, pin_v, pin_f, out_f

    # --- the other factor precisions of the same workload (same protocol, fewer steps)
    var_out = {}
    for vdt in variants:
        _, vc, vv, vinit, vfac = inputs(vdt)
        vstep = make_step(vdt, vc, vv, vfac, vinit)
        vres, _ = vstep()
        torch.cuda.synchronize()
        vsteps = max(1, min(args.steps, 3))
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(vsteps):
            vres, _ = vstep()
        a1.record(stream)
        torch.cuda.synchronize()
        vms = _max_over_ranks(dist, a0.elapsed_time(a1))
        hv = rl.relate_encode(vc, vv, spec.dims, factor_dtype=vdt, stream=stream)
        _, vper = _time_kernels(rl, torch, hv, stream, vfac, spec, R, vdt, dev, 3)
        hv.close()
        var_out[vdt] = {"value": units_step * vsteps * world / (vms / 1000.0), "unit": UNIT,
                        "ms_per_step": vms / vsteps, "steps": vsteps, "dtype": "f32",
                        "final_fit": vres["fit"], "roofline": _roofline(vper, vdt, spec.name, spec.nnz)}
        del vc, vv, vinit, vfac

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f64" if fdt == "f64" else "f32",
            "data": "synthetic",
            "config": {**wcfg(fdt), "parallelism": (f"nnz-shards{world}" if sharded else f"replicas{world}")
                       if world > 1 else "single",
                       "step": f"encode + {iters} CP-ALS iterations (tol 0), one CUDA graph per iteration",
                       "l2": "inputs larger than L2 (stream %d MB); L2 flushed between kernel timings"
                             % (spec.nnz * (stats['key_bytes'] + (8 if fdt == 'f64' else 4)) // 2 ** 20),
                       "final_fit": res["fit"]},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": _launches_per_step(stats, iters, fdt, sum(1 for m in per_mode if m["strategy"] == 2),
                                               R, [m["kr_pair"] for m in per_mode]) * args.steps,
            "roofline": roof,
            "clocks": clk.summary()}
    if var_out:
        line["variants"] = var_out
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, coords, vals)
    if rank == 0:
        print(f"# generation {t_gen:.1f} s; per-mode MTTKRP ms {[round(m['ms'], 3) for m in per_mode]}",
              file=sys.stderr)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
