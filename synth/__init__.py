"""Seeded synthetic sparse tensors and factor initialisations.

This module is shared by the CPU oracle's tests and the CUDA path's tests and
benchmark. It holds NO arithmetic of the method (no encoding, no MTTKRP, no
ALS): only counter-based random numbers and the distributions built on them.

Random numbers: SplitMix64 (Steele, Lea & Flood, 2014) in counter mode. The
draw for (seed, tag, index) is ``mix64(base + (index + 1) * GAMMA)`` with
``base = mix64(seed * GAMMA + tag)``; so every array is deterministic and can
be generated in any order or in parallel.

Distributions:
* uniform(0,1]   = ((x >> 11) + 1) * 2^-53.
* uniform label on [0, I) = floor(((x >> 11) * 2^-53) * I).
* Zipf(alpha) on [0, I): P(k) proportional to (k+1)^-alpha, by inverse CDF
  (binary search in an FP64 cumulative table).
* lognormal(0,1) = exp(z), z from Box-Muller on two uniform(0,1] draws, FP64,
  then rounded to FP32.
* "shuffled" labels: a seeded per-mode permutation of [0, I) (the paper's
  shuffled experiments, Sec. 4.1.3).
* Distinct coordinates: draws are taken in counter order and the first
  occurrence of each coordinate tuple is kept until nnz tuples are collected.

The tensors stand in for the FROSTT tensors of the paper's Table I (not
available here): power-law modes, a short time-like mode, hyper-sparse dims.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_C_LIB = None
_C_LOCK = threading.Lock()


def _clib():
    """The multithreaded C helper (synthc.c), compiled on first use; None if
    no compiler is available (the numpy path then runs)."""
    global _C_LIB
    with _C_LOCK:
        if _C_LIB is None:
            src = os.path.join(_HERE, "synthc.c")
            out = os.path.join(_HERE, "_build", "libsynthc.so")
            try:
                os.makedirs(os.path.dirname(out), exist_ok=True)
                if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
                    tmp = out + f".tmp{os.getpid()}"
                    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp],
                                   check=True, capture_output=True)
                    os.replace(tmp, out)
                L = ctypes.CDLL(out)
                P, I64, U64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
                L.synth_base.restype, L.synth_base.argtypes = U64, [U64, U64]
                L.synth_labels.restype = None
                L.synth_labels.argtypes = [U64, I64, I64, I, U64, P, P, P, I]
                L.synth_dedup_new.restype, L.synth_dedup_new.argtypes = P, [I, P, I, U64, I]
                L.synth_dedup_free.restype, L.synth_dedup_free.argtypes = None, [P]
                L.synth_dedup_insert.restype, L.synth_dedup_insert.argtypes = I64, [P, P, I64, P]
                _C_LIB = L
            except Exception:
                _C_LIB = False
        return _C_LIB or None


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return os.cpu_count() or 1

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TAG_COORD = 0x100   # + mode
TAG_VAL = 0x200
TAG_VAL2 = 0x201
TAG_FACTOR = 0x300
TAG_LABELS = 0x400  # + mode
TAG_REQUEST = 0x500
TAG_ARRIVAL = 0x600


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream(seed: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Counter-mode SplitMix64 draws for indices idx (uint64)."""
    with np.errstate(over="ignore"):
        base = mix64(np.array([(seed * 0x9E3779B97F4A7C15 + tag) & (2**64 - 1)], dtype=np.uint64))[0]
        idx = np.asarray(idx, dtype=np.uint64)
        return mix64(base + (idx + np.uint64(1)) * GAMMA)


def uniform01(x: np.ndarray) -> np.ndarray:
    """uniform(0,1] from 64-bit draws."""
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def uniform_label(x: np.ndarray, I: int) -> np.ndarray:
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.minimum((u * I).astype(np.int64), I - 1).astype(np.uint32)


def zipf_table(I: int, alpha: float) -> np.ndarray:
    w = np.arange(1, I + 1, dtype=np.float64) ** (-float(alpha))
    return np.cumsum(w)


def zipf_label(x: np.ndarray, cdf: np.ndarray) -> np.ndarray:
    t = uniform01(x) * cdf[-1]
    k = np.searchsorted(cdf, t, side="left")
    return np.minimum(k, len(cdf) - 1).astype(np.uint32)


def label_permutation(seed: int, mode: int, I: int) -> np.ndarray:
    keys = stream(seed, TAG_LABELS + mode, np.arange(I, dtype=np.uint64))
    return np.argsort(keys, kind="stable").astype(np.uint32)


@dataclass
class TensorSpec:
    """A synthetic sparse tensor: dims, nnz, per-mode label distribution."""
    name: str
    dims: tuple
    nnz: int
    dists: tuple            # per mode: ("uniform",) or ("zipf", alpha)
    values: str = "uniform"  # "uniform" (U(0,1]) or "lognormal"
    value_dtype: str = "f32"  # "f32" or "f64"
    seed: int = 1
    shuffle: bool = False
    distinct: bool | str = True   # True, False, or "once" (see make_tensor)
    extra: dict = field(default_factory=dict)


def _draw_coords(spec: TensorSpec, lo: int, hi: int, tables, use_c: bool = True) -> np.ndarray:
    N = len(spec.dims)
    out = np.empty((N, hi - lo), dtype=np.uint32)
    L = _clib() if use_c else None
    if L is not None:
        for n in range(N):
            d = spec.dists[n]
            cdf = tables[n] if d[0] == "zipf" else None
            perm = tables[N + n] if spec.shuffle else None
            base = L.synth_base(spec.seed, TAG_COORD + n)
            L.synth_labels(base, lo, hi - lo, 1 if d[0] == "zipf" else 0, int(spec.dims[n]),
                           cdf.ctypes.data if cdf is not None else None,
                           perm.ctypes.data if perm is not None else None, out[n].ctypes.data, _threads())
        return out
    idx = np.arange(lo, hi, dtype=np.uint64)
    for n in range(N):
        x = stream(spec.seed, TAG_COORD + n, idx)
        d = spec.dists[n]
        if d[0] == "zipf":
            lab = zipf_label(x, tables[n])
        elif d[0] == "uniform":
            lab = uniform_label(x, int(spec.dims[n]))
        else:
            raise ValueError(f"unknown distribution {d}")
        if spec.shuffle:
            lab = tables[N + n][lab]
        out[n] = lab
    return out


def _dedup_keys(coords: np.ndarray, dims) -> list:
    """Split the modes into groups whose mixed-radix products fit in uint64
    and return one uint64 key per group (most significant group first)."""
    groups, cur, prod = [], [], 1
    for n, I in enumerate(dims):
        if prod * int(I) >= 2 ** 64:
            groups.append(cur)
            cur, prod = [], 1
        cur.append(n)
        prod *= int(I)
    groups.append(cur)
    keys = []
    for g in groups:
        k = np.zeros(coords.shape[1], dtype=np.uint64)
        with np.errstate(over="ignore"):
            for n in g:
                k = k * np.uint64(int(dims[n])) + coords[n].astype(np.uint64)
        keys.append(k)
    return keys


def _split_point(dims) -> int:
    """Modes [0, split) and [split, N) each have a mixed-radix product < 2^64."""
    prod, split = 1, 0
    for n, I in enumerate(dims):
        if prod * int(I) >= 2 ** 64:
            break
        prod *= int(I)
        split = n + 1
    rest = 1
    for I in dims[split:]:
        rest *= int(I)
    if rest >= 2 ** 64:
        raise ValueError("tensor too large for the distinct-coordinate check")
    return split


def _make_coords_c(spec: TensorSpec, tables, L) -> np.ndarray | None:
    N = len(spec.dims)
    dims = np.array(spec.dims, dtype=np.uint64)
    T = _threads()
    st = L.synth_dedup_new(N, dims.ctypes.data, _split_point(spec.dims), 2 * spec.nnz + 4096, T)
    if not st:
        return None
    try:
        kept_parts, have, cursor = [], 0, 0
        batch = int(spec.nnz * 1.1) + 1024
        for _ in range(200):
            c = _draw_coords(spec, cursor, cursor + batch, tables)
            cursor += batch
            keep = np.zeros(batch, dtype=np.uint8)
            if L.synth_dedup_insert(st, c.ctypes.data, batch, keep.ctypes.data) < 0 or (keep == 2).any():
                return None
            idx = np.nonzero(keep)[0][: spec.nnz - have]
            kept_parts.append(c[:, idx])
            have += idx.shape[0]
            if have >= spec.nnz:
                return np.ascontiguousarray(np.concatenate(kept_parts, axis=1))
            batch = max(int((spec.nnz - have) * 2.0), 1024)
        raise ValueError(f"{spec.name}: could not draw {spec.nnz} distinct coordinates")
    finally:
        L.synth_dedup_free(st)


def make_coords(spec: TensorSpec, use_c: bool = True) -> np.ndarray:
    N = len(spec.dims)
    tables = []
    for n in range(N):
        d = spec.dists[n]
        tables.append(zipf_table(int(spec.dims[n]), d[1]) if d[0] == "zipf" else None)
    if spec.shuffle:
        for n in range(N):
            tables.append(label_permutation(spec.seed, n, int(spec.dims[n])))
    if not spec.distinct:
        return _draw_coords(spec, 0, spec.nnz, tables, use_c)
    L = _clib() if use_c else None
    if L is not None:
        got = _make_coords_c(spec, tables, L)
        if got is not None:
            return got
    # Take draws in counter order, keeping the first occurrence of each tuple,
    # in batches; `seen` holds the kept tuples' keys sorted for lookups.
    kept_parts, seen, have, cursor = [], None, 0, 0
    batch = int(spec.nnz * 1.1) + 1024
    for _ in range(200):
        c = _draw_coords(spec, cursor, cursor + batch, tables, use_c=False)
        cursor += batch
        keys = _dedup_keys(c, spec.dims)
        if len(keys) == 1:
            k = keys[0]
        else:  # pack (hi, lo) into a structured view comparable as a pair
            k = np.empty(c.shape[1], dtype=[("h", np.uint64), ("l", np.uint64)])
            k["h"], k["l"] = keys[0], keys[1] if len(keys) == 2 else _fold(keys[1:])
        order = np.argsort(k, kind="stable")
        ks = k[order]
        first = np.ones(c.shape[1], dtype=bool)
        first[order[1:][ks[1:] == ks[:-1]]] = False
        if seen is not None:
            pos = np.searchsorted(seen, k)
            pos = np.minimum(pos, len(seen) - 1)
            first &= seen[pos] != k
        idx = np.nonzero(first)[0][: spec.nnz - have]
        kept_parts.append(c[:, idx])
        have += idx.shape[0]
        if have >= spec.nnz:
            return np.ascontiguousarray(np.concatenate(kept_parts, axis=1))
        seen = np.sort(k[idx]) if seen is None else np.sort(np.concatenate([seen, k[idx]]))
        batch = max(int((spec.nnz - have) * 2.0), 1024)
    raise ValueError(f"{spec.name}: could not draw {spec.nnz} distinct coordinates")


def _fold(keys):
    if len(keys) != 1:
        raise ValueError("tensor too large for the distinct-coordinate check")
    return keys[0]


def make_values(spec: TensorSpec) -> np.ndarray:
    idx = np.arange(spec.nnz, dtype=np.uint64)
    u1 = uniform01(stream(spec.seed, TAG_VAL, idx))
    if spec.values == "uniform":
        v = u1
    elif spec.values == "lognormal":
        u2 = uniform01(stream(spec.seed, TAG_VAL2, idx))
        v = np.exp(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2))
    elif spec.values.startswith("int"):
        # "int:a:b" -> integers uniform in [a, b] (exact-arithmetic cases)
        _, a, b = spec.values.split(":")
        a, b = int(a), int(b)
        v = (a + np.minimum((u1 * (b - a + 1)).astype(np.int64), b - a)).astype(np.float64)
    else:
        raise ValueError(spec.values)
    return v.astype(np.float32) if spec.value_dtype == "f32" else v.astype(np.float64)


def _distinct_once(spec: TensorSpec) -> tuple[np.ndarray, np.ndarray]:
    """Draws spec.nnz tuples once and keeps the first occurrence of each
    distinct tuple (no top-up): returns (coords, indices of the kept draws)."""
    N = len(spec.dims)
    tables = [zipf_table(int(I), d[1]) if d[0] == "zipf" else None for I, d in zip(spec.dims, spec.dists)]
    if spec.shuffle:
        tables += [label_permutation(spec.seed, n, int(spec.dims[n])) for n in range(N)]
    c = _draw_coords(spec, 0, spec.nnz, tables)
    L = _clib()
    if L is not None and spec.nnz > 0:
        dims = np.array(spec.dims, dtype=np.uint64)
        st = L.synth_dedup_new(N, dims.ctypes.data, _split_point(spec.dims), 2 * spec.nnz + 4096, _threads())
        if st:
            try:
                keep = np.zeros(spec.nnz, dtype=np.uint8)
                if L.synth_dedup_insert(st, c.ctypes.data, spec.nnz, keep.ctypes.data) >= 0 and not (keep == 2).any():
                    idx = np.nonzero(keep)[0]
                    return np.ascontiguousarray(c[:, idx]), idx
            finally:
                L.synth_dedup_free(st)
    keys = _dedup_keys(c, spec.dims)
    order = np.lexsort(keys[::-1]) if c.shape[1] else np.zeros(0, dtype=np.int64)
    first = np.ones(c.shape[1], dtype=bool)
    if c.shape[1] > 1:
        same = np.ones(c.shape[1] - 1, dtype=bool)
        for k in keys:
            ks = k[order]
            same &= ks[1:] == ks[:-1]
        first[order[1:][same]] = False  # lexsort is stable: the first draw stays
    idx = np.nonzero(first)[0]
    return np.ascontiguousarray(c[:, idx]), idx


def make_tensor(spec: TensorSpec):
    """Returns (coords (N, nnz) uint32 SoA, vals (nnz,) f32/f64). With
    distinct == "once", spec.nnz tuples are drawn once and repeats dropped
    (the tensor then has at most spec.nnz nonzeros)."""
    if spec.distinct == "once":
        c, idx = _distinct_once(spec)
        return c, make_values(spec)[idx]
    return make_coords(spec), make_values(spec)


def init_factors(dims, R: int, seed: int = 0, dtype=np.float64, kind: str = "uniform"):
    """Factor initialisation: uniform(0,1] drawn in order (mode k, row i,
    column r) from one counter stream; FP64, then rounded to dtype.
    kind="int:a:b" draws integers in [a, b] instead (exact cases)."""
    out, off = [], 0
    for I in dims:
        idx = np.arange(off, off + int(I) * R, dtype=np.uint64)
        u = uniform01(stream(seed, TAG_FACTOR, idx))
        if kind.startswith("int"):
            _, a, b = kind.split(":")
            a, b = int(a), int(b)
            u = (a + np.minimum((u * (b - a + 1)).astype(np.int64), b - a)).astype(np.float64)
        out.append(u.reshape(int(I), R).astype(dtype))
        off += int(I) * R
    return out


# ----------------------------------------------------------------------------
# Named workloads (the sizes the paper's workloads are stood in by)
# ----------------------------------------------------------------------------
WORKLOADS = {
    # plain FP64 CP-ALS: 1000^3, 1M uniform distinct coords, U(0,1] values
    "uniform3d-1000x1000x1000-1M": dict(
        spec=TensorSpec("uniform3d-1000x1000x1000-1M", (1000, 1000, 1000), 1_000_000,
                        (("uniform",),) * 3, values="uniform", value_dtype="f64", seed=1),
        R=16, iters=10, factor_dtype="f64"),
    # skewed 3-mode: Zipf 1.2 on every mode, lognormal FP32 values
    "zipf3d-200Kx200Kx5K-50M": dict(
        spec=TensorSpec("zipf3d-200Kx200Kx5K-50M", (200_000, 200_000, 5_000), 50_000_000,
                        (("zipf", 1.2),) * 3, values="lognormal", value_dtype="f32", seed=2),
        R=32, iters=25, factor_dtype="f32"),
    # the same recipe at 20M nonzeros (stream 240 MB > L2): small case for profiler captures
    "zipf3d-200Kx200Kx5K-20M": dict(
        spec=TensorSpec("zipf3d-200Kx200Kx5K-20M", (200_000, 200_000, 5_000), 20_000_000,
                        (("zipf", 1.2),) * 3, values="lognormal", value_dtype="f32", seed=2),
        R=32, iters=25, factor_dtype="f32"),
    # 4-mode with a short time-like mode
    "zipf4d-5Mx1Mx100Kx24-150M": dict(
        spec=TensorSpec("zipf4d-5Mx1Mx100Kx24-150M", (5_000_000, 1_000_000, 100_000, 24),
                        150_000_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                        values="uniform", value_dtype="f32", seed=3),
        R=64, iters=10, factor_dtype="f32"),
    # the same recipe at 30M nonzeros: small case for profiler captures
    "zipf4d-5Mx1Mx100Kx24-30M": dict(
        spec=TensorSpec("zipf4d-5Mx1Mx100Kx24-30M", (5_000_000, 1_000_000, 100_000, 24),
                        30_000_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                        values="uniform", value_dtype="f32", seed=3),
        R=64, iters=10, factor_dtype="f32"),
    # 5-mode hyper-sparse
    "zipf5d-10Mx10Mx1Mx1Kx100-100M": dict(
        spec=TensorSpec("zipf5d-10Mx10Mx1Mx1Kx100-100M", (10_000_000, 10_000_000, 1_000_000, 1000, 100),
                        100_000_000, (("zipf", 1.3),) * 2 + (("uniform",),) * 3,
                        values="uniform", value_dtype="f32", seed=4),
        R=16, iters=10, factor_dtype="bf16"),
    # the 5-mode recipe at 20M nonzeros: small case for profiler captures
    "zipf5d-10Mx10Mx1Mx1Kx100-20M": dict(
        spec=TensorSpec("zipf5d-10Mx10Mx1Mx1Kx100-20M", (10_000_000, 10_000_000, 1_000_000, 1000, 100),
                        20_000_000, (("zipf", 1.3),) * 2 + (("uniform",),) * 3,
                        values="uniform", value_dtype="f32", seed=4),
        R=16, iters=10, factor_dtype="bf16"),
}


def scaled(spec: TensorSpec, nnz: int, dims=None, name: str | None = None) -> TensorSpec:
    """The same recipe at a smaller size (for parity cases)."""
    return TensorSpec(name or f"{spec.name}@{nnz}", tuple(dims or spec.dims), nnz, spec.dists,
                      spec.values, spec.value_dtype, spec.seed, spec.shuffle, spec.distinct)


def _log_uniform(u: float, lo: float, hi: float) -> float:
    return math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def _pick(u: float, choices):
    return choices[min(int(u * len(choices)), len(choices) - 1)]


def serving_request(i: int, seed_base: int = 1000, nnz_range=(1e4, 2e7), dim_range=(100, 1e6),
                    alpha_range=(1.0, 1.4), ranks=(8, 16, 32, 64), modes=(3, 4, 5)):
    """Request i of the serving mix (the decomposition requests of a
    CP-ALS service): seed = seed_base + i; N uniform over `modes`; nnz and
    every I_n log-uniform over their ranges; one Zipf exponent for all modes,
    uniform over alpha_range; R uniform over `ranks`; U(0,1] FP32 values.
    nnz tuples are drawn once and repeated tuples dropped (first draw kept),
    since a Zipf law on 100-long modes cannot supply millions of distinct
    tuples: the tensor has at most nnz nonzeros. Returns (TensorSpec, R)."""
    seed = seed_base + int(i)
    u = uniform01(stream(seed, TAG_REQUEST, np.arange(16, dtype=np.uint64)))
    N = _pick(u[0], modes)
    nnz = int(round(_log_uniform(u[1], *nnz_range)))
    dims = tuple(int(round(_log_uniform(u[2 + n], *dim_range))) for n in range(N))
    alpha = alpha_range[0] + u[12] * (alpha_range[1] - alpha_range[0])
    R = _pick(u[13], ranks)
    spec = TensorSpec(f"serve-{i}", dims, nnz, (("zipf", float(alpha)),) * N, values="uniform",
                      value_dtype="f32", seed=seed, distinct="once")
    return spec, R


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate:
    cumulative sums of exponential gaps -ln(u) / rate."""
    u = uniform01(stream(seed, TAG_ARRIVAL, np.arange(n, dtype=np.uint64)))
    return np.cumsum(-np.log(u) / float(rate))

