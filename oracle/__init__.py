"""CPU oracle for the ReLATE hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
library (``paper_2509_00280_gb300``) never imports, links or calls it, and the
two share no code, header or constant table.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, FP64, 128-bit
positions); this module only compiles it with gcc and marshals numpy arrays.
Each wrapper names the paper passage its C function follows:

* ``bit_budget`` / ``alto_order`` / ``check_order`` -- Sec. 3.3, 3.3.1-3.3.2,
  Fig. 4, and the masking rule of Alg. 1 (Sec. 3.4).
* ``encode`` / ``decode`` / ``sort_perm`` -- Sec. 3.3 (linearized tensor
  ordered by position p; bit-level encode/decode).
* ``partitions`` / ``mode_stats`` -- equal-work partitions (Sec. 4.2) and fiber
  reuse statistics (Sec. 4.1.3).
* ``mttkrp`` -- Sec. 2.2 and Fig. 2 (per-nonzero MTTKRP), Neumaier-compensated.
* ``cpals`` and helpers -- standard CP-ALS (Kolda & Bader, cited in Sec. 2.2).

Parity unpinned: the ALTO tie-break between equal-length modes beyond the
paper's 4x8x2 example; the exact ALS variant of the paper's TD library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_ORDER, ERR_WIDE, ERR_RANGE, ERR_NOT_PD, ERR_OOM = 0, -1, -2, -3, -4, -5, -6


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so with gcc (portable flags)
    (and oracle_omp.c, the CPU baseline's OpenMP MTTKRP)."""
    build_omp(force)
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_OMP_SRC = os.path.join(_HERE, "oracle_omp.c")
_OMP_LIB = os.path.join(_OUT_DIR, "liboracle_omp.so")
_omp_lib = None


def build_omp(force: bool = False) -> str:
    """Compile oracle_omp.c (the OpenMP MTTKRP of the CPU baseline) with
    -O3 -fopenmp, and -mcpu=native on an aarch64 host; FP contraction off, as
    for the oracle itself."""
    import platform
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_OMP_LIB)) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_OMP_SRC)
    if force or stale:
        tmp = _OMP_LIB + f".tmp{os.getpid()}"
        cpu = ["-mcpu=native"] if platform.machine() in ("aarch64", "arm64") else []
        cmd = ["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", *cpu,
               _OMP_SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


def _load_omp():
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            build_omp()
            lib = ctypes.CDLL(_OMP_LIB)
            P = ctypes.c_void_p
            lib.orc_omp_max_threads.restype, lib.orc_omp_max_threads.argtypes = ctypes.c_int, []
            lib.orc_mttkrp_omp.restype = ctypes.c_int
            lib.orc_mttkrp_omp.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P,
                                           ctypes.c_int, ctypes.c_int64]
            _omp_lib = lib
    return _omp_lib


def mttkrp_omp(coords: np.ndarray, vals: np.ndarray, dims, mode: int, factors, nthreads: int,
               priv_limit: int = 4 * 1024 * 1024, out: np.ndarray | None = None) -> np.ndarray:
    """OpenMP MTTKRP for the CPU baseline's timing (oracle_omp.c): the
    oracle's per-nonzero arithmetic over nthreads contiguous nonzero chunks;
    per-thread output copies when I_n x R <= priv_limit, else atomics. Not a
    correctness reference (its sums are not compensated)."""
    c = _c(coords, np.uint32)
    v = _c(vals, np.float64)
    d = _c(dims, np.uint64)
    N, nnz = c.shape
    fs = [_c(f, np.float64) for f in factors]
    R = fs[0].shape[1]
    ptrs = (ctypes.c_void_p * N)(*[_p(f) for f in fs])
    if out is None:
        out = np.empty((int(d[mode]), R), dtype=np.float64)
    _check(_load_omp().orc_mttkrp_omp(_p(c), _p(v), _p(d), nnz, N, mode, ptrs, R, _p(out), int(nthreads),
                                      int(priv_limit)), "mttkrp_omp")
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_bits_for_dim": (i32, [u64]),
                "orc_bit_budget": (i32, [P, i32, P]),
                "orc_check_order": (i32, [P, i32, P, i32]),
                "orc_alto_order": (i32, [P, i32, P]),
                "orc_encode": (i32, [P, P, i64, i32, P, P, P]),
                "orc_decode": (i32, [P, P, P, i64, i32, P, P]),
                "orc_sort_perm": (None, [P, P, i64, P]),
                "orc_partitions": (i64, [P, i64, i32, i64, P, P]),
                "orc_mode_stats": (i32, [P, P, i64, i32, i64, P, P, P, P]),
                "orc_mttkrp": (i32, [P, P, P, i64, i32, i32, P, i32, P]),
                "orc_gram": (None, [P, u64, i32, P]),
                "orc_cholesky": (i32, [P, i32, P]),
                "orc_solve_rows": (None, [P, u64, i32, P, P]),
                "orc_factor_normal": (i32, [P, i32, P, P]),
                "orc_cpals": (i32, [P, P, P, i64, i32, i32, i32, f64, P, P, P, P, P]),
                "orc_round_bf16": (None, [P, i64, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise OracleError(f"{what}: oracle status {rc}")


# --------------------------------------------------------------------------
# Encoding (Sec. 3.3)
# --------------------------------------------------------------------------
def bits_for_dim(I: int) -> int:
    return int(_load().orc_bits_for_dim(int(I)))


def bit_budget(dims) -> tuple[list[int], int]:
    d = _c(dims, np.uint64)
    lb = np.zeros(len(d), dtype=np.int32)
    lp = _load().orc_bit_budget(_p(d), len(d), _p(lb))
    return [int(x) for x in lb], int(lp)


def check_order(dims, order) -> bool:
    d = _c(dims, np.uint64)
    o = _c(order, np.int8)
    return _load().orc_check_order(_p(d), len(d), _p(o), len(o)) == OK


def alto_order(dims) -> np.ndarray:
    d = _c(dims, np.uint64)
    _, lp = bit_budget(d)
    o = np.zeros(max(lp, 1), dtype=np.int8)
    _load().orc_alto_order(_p(d), len(d), _p(o))
    return o[:lp].copy()


def encode(coords: np.ndarray, dims, order) -> tuple[np.ndarray, np.ndarray]:
    """coords: (N, nnz) uint32. Returns (key_lo, key_hi) uint64 arrays of p."""
    c = _c(coords, np.uint32)
    d = _c(dims, np.uint64)
    o = _c(order, np.int8)
    N, nnz = c.shape
    lo = np.zeros(nnz, dtype=np.uint64)
    hi = np.zeros(nnz, dtype=np.uint64)
    _check(_load().orc_encode(_p(c), _p(d), nnz, N, _p(o), _p(lo), _p(hi)), "encode")
    return lo, hi


def decode(key_lo, key_hi, dims, order) -> np.ndarray:
    lo = _c(key_lo, np.uint64)
    hi = _c(key_hi, np.uint64)
    d = _c(dims, np.uint64)
    o = _c(order, np.int8)
    nnz = lo.shape[0]
    out = np.zeros((len(d), nnz), dtype=np.uint32)
    _check(_load().orc_decode(_p(lo), _p(hi), _p(d), nnz, len(d), _p(o), _p(out)), "decode")
    return out


def sort_perm(key_lo, key_hi) -> np.ndarray:
    lo = _c(key_lo, np.uint64)
    hi = _c(key_hi, np.uint64)
    perm = np.zeros(lo.shape[0], dtype=np.uint32)
    _load().orc_sort_perm(_p(lo), _p(hi), lo.shape[0], _p(perm))
    return perm


def partitions(coords_sorted: np.ndarray, S: int) -> tuple[np.ndarray, np.ndarray]:
    c = _c(coords_sorted, np.uint32)
    N, nnz = c.shape
    P = (nnz + S - 1) // S
    lo = np.zeros((max(P, 1), N), dtype=np.uint32)
    hi = np.zeros((max(P, 1), N), dtype=np.uint32)
    got = _load().orc_partitions(_p(c), nnz, N, S, _p(lo), _p(hi))
    if got < 0:
        raise OracleError(f"partitions: status {got}")
    return lo[:P].copy(), hi[:P].copy()


def mode_stats(coords_sorted: np.ndarray, dims, S: int, with_counts: bool = False):
    c = _c(coords_sorted, np.uint32)
    d = _c(dims, np.uint64)
    N, nnz = c.shape
    runs = np.zeros(N, dtype=np.uint64)
    distinct = np.zeros(N, dtype=np.uint64)
    maxcount = np.zeros(N, dtype=np.uint64)
    counts = np.zeros(int(d.sum()) if with_counts else 1, dtype=np.uint64)
    _check(_load().orc_mode_stats(_p(c), _p(d), nnz, N, S, _p(runs), _p(distinct),
                                  _p(maxcount), _p(counts) if with_counts else None),
           "mode_stats")
    out = {"runs": runs, "distinct": distinct, "maxcount": maxcount}
    if with_counts:
        parts, off = [], 0
        for n in range(N):
            parts.append(counts[off:off + int(d[n])].copy())
            off += int(d[n])
        out["counts"] = parts
    return out


def encode_full(coords: np.ndarray, vals: np.ndarray, dims, order=None, S: int = 4096):
    """The whole encoding step: positions, stable sort, partitions, stats."""
    if order is None:
        order = alto_order(dims)
    lo, hi = encode(coords, dims, order)
    perm = sort_perm(lo, hi)
    cs = np.ascontiguousarray(np.asarray(coords, dtype=np.uint32)[:, perm])
    plo, phi = partitions(cs, S)
    st = mode_stats(cs, dims, S)
    return {"order": np.asarray(order, dtype=np.int8), "key_lo": lo[perm], "key_hi": hi[perm],
            "perm": perm, "coords": cs, "vals": np.asarray(vals)[perm], "part_lo": plo,
            "part_hi": phi, **st}


# --------------------------------------------------------------------------
# MTTKRP (Sec. 2.2, Fig. 2)
# --------------------------------------------------------------------------
def mttkrp(coords: np.ndarray, vals: np.ndarray, dims, mode: int, factors) -> np.ndarray:
    c = _c(coords, np.uint32)
    v = _c(vals, np.float64)
    d = _c(dims, np.uint64)
    N, nnz = c.shape
    fs = [_c(f, np.float64) for f in factors]
    R = fs[0].shape[1]
    ptrs = (ctypes.c_void_p * N)(*[_p(f) for f in fs])
    out = np.zeros((int(d[mode]), R), dtype=np.float64)
    _check(_load().orc_mttkrp(_p(c), _p(v), _p(d), nnz, N, mode, ptrs, R, _p(out)), "mttkrp")
    return out


# --------------------------------------------------------------------------
# Dense CP-ALS remainder (standard ALS)
# --------------------------------------------------------------------------
def gram(A: np.ndarray) -> np.ndarray:
    a = _c(A, np.float64)
    I, R = a.shape
    G = np.zeros((R, R), dtype=np.float64)
    _load().orc_gram(_p(a), I, R, _p(G))
    return G


def cholesky(V: np.ndarray) -> np.ndarray:
    v = _c(V, np.float64)
    R = v.shape[0]
    L = np.zeros((R, R), dtype=np.float64)
    _check(_load().orc_cholesky(_p(v), R, _p(L)), "cholesky")
    return L


def factor_normal(V: np.ndarray) -> tuple[np.ndarray, int]:
    """Cholesky of the normal-equations matrix with the oracle's one ridge
    retry (V + 1e-12 tr(V)/R I when V itself fails). Returns (L, ridged)."""
    v = _c(V, np.float64)
    R = v.shape[0]
    L = np.zeros((R, R), dtype=np.float64)
    ridged = ctypes.c_int(0)
    _check(_load().orc_factor_normal(_p(v), R, _p(L), ctypes.byref(ridged)), "factor_normal")
    return L, int(ridged.value)


def solve_rows(M: np.ndarray, V: np.ndarray) -> np.ndarray:
    """A = M V^{-1} through the oracle's Cholesky (with ridge retry)."""
    m = _c(M, np.float64)
    v = _c(V, np.float64)
    I, R = m.shape
    L = np.zeros((R, R), dtype=np.float64)
    ridged = ctypes.c_int(0)
    _check(_load().orc_factor_normal(_p(v), R, _p(L), ctypes.byref(ridged)), "factor_normal")
    A = np.zeros_like(m)
    _load().orc_solve_rows(_p(m), I, R, _p(L), _p(A))
    return A


def cpals(coords, vals, dims, R: int, iters: int, tol: float, factors):
    """Returns dict(factors, lam, fit_trace, iters, ridges). factors are
    copied; the inputs are not modified."""
    c = _c(coords, np.uint32)
    v = _c(vals, np.float64)
    d = _c(dims, np.uint64)
    N, nnz = c.shape
    fs = [np.array(f, dtype=np.float64, copy=True, order="C") for f in factors]
    ptrs = (ctypes.c_void_p * N)(*[_p(f) for f in fs])
    lam = np.zeros(R, dtype=np.float64)
    trace = np.zeros(max(iters, 1), dtype=np.float64)
    done = ctypes.c_int(0)
    ridges = ctypes.c_int(0)
    rc = _load().orc_cpals(_p(c), _p(v), _p(d), nnz, N, R, iters, float(tol), ptrs, _p(lam),
                           _p(trace), ctypes.byref(done), ctypes.byref(ridges))
    _check(rc, "cpals")
    return {"factors": fs, "lam": lam, "fit_trace": trace[:done.value].copy(),
            "iters": done.value, "ridges": ridges.value}


def round_bf16(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 round-to-nearest-even, returned as FP32 values."""
    a = _c(x, np.float32)
    out = np.empty_like(a)
    _load().orc_round_bf16(_p(a), a.size, _p(out))
    return out
