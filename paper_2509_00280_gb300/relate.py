"""ctypes binding of include/relate.h -- argument marshalling only.

Function names follow the C ABI. Device pointers come from torch CUDA
tensors (``tensor.data_ptr()``), host pointers from numpy arrays, streams
from ``torch.cuda.Stream`` (``.cuda_stream``) or raw integers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_build", "librelate.so")

RELATE_F64, RELATE_F32, RELATE_BF16 = 0, 1, 2
RELATE_CONFLICT_AUTO, RELATE_CONFLICT_ATOMIC, RELATE_CONFLICT_SEGMENTED, RELATE_CONFLICT_PRIVATIZED = 0, 1, 2, 3
MAX_MODES, MAX_RANK, MAX_KEY_BITS = 8, 64, 128

_DTYPES = {"f64": RELATE_F64, "f32": RELATE_F32, "bf16": RELATE_BF16,
           RELATE_F64: RELATE_F64, RELATE_F32: RELATE_F32, RELATE_BF16: RELATE_BF16}


class RelateError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {relate_status_string(status)} ({status}): {relate_last_error()}")


class Params(ctypes.Structure):
    _fields_ = [("bit_order", ctypes.c_void_p), ("bit_order_len", ctypes.c_int),
                ("partition_size", ctypes.c_int64), ("conflict", ctypes.c_int * MAX_MODES),
                ("val_dtype", ctypes.c_int), ("factor_dtype", ctypes.c_int), ("acc_dtype", ctypes.c_int),
                ("coords_on_device", ctypes.c_int), ("stream", ctypes.c_void_p), ("smem_budget", ctypes.c_int),
                ("shard_rank", ctypes.c_int), ("shard_count", ctypes.c_int)]


class CpalsInfo(ctypes.Structure):
    _fields_ = [("fit", ctypes.c_double), ("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("ridge_retries", ctypes.c_int), ("fit_trace", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int), ("lp", ctypes.c_int), ("key_bytes", ctypes.c_int),
                ("nnz", ctypes.c_int64), ("partition_size", ctypes.c_int64), ("partitions", ctypes.c_int64),
                ("dims", ctypes.c_uint64 * MAX_MODES), ("lbits", ctypes.c_int * MAX_MODES),
                ("field_offset", ctypes.c_int * MAX_MODES), ("runs", ctypes.c_uint64 * MAX_MODES),
                ("distinct", ctypes.c_uint64 * MAX_MODES), ("maxcount", ctypes.c_uint64 * MAX_MODES),
                ("bit_order", ctypes.c_int8 * MAX_KEY_BITS), ("nnz_total", ctypes.c_int64), ("shard_lo", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Loads librelate.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"librelate.so is not built ({_LIB_PATH}); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(_LIB_PATH)
            P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "relate_params_default": (None, [P]),
                "relate_encode": (I, [P, P, P, I, I64, P, P]),
                "relate_mttkrp": (I, [P, I, P, I, P, P]),
                "relate_cpals": (I, [P, I, I, D, P, P, P]),
                "relate_get_stats": (I, [P, P]),
                "relate_get_conflict": (I, [P, I, I, P]),
                "relate_set_conflict": (I, [P, I, I]),
                "relate_set_precision": (I, [P, I, I]),
                "relate_set_mode_plan": (I, [P, I, I, P, I]),
                "relate_mttkrp_batch": (I, [P, I, P]),
                "relate_shard_range": (None, [I64, I, I, P, P]),
                "relate_set_reduce_hook": (I, [P, P, P]),
                "relate_cpals_batch": (I, [P, I, P, I, D, P, P, P, P, P]),
                "relate_get_mode_plan": (I, [P, I, I, P, P, P]),
                "relate_set_mode_kr": (I, [P, I, I]),
                "relate_get_mode_kr": (I, [P, I, I, P, P]),
                "relate_set_stream": (I, [P, P]),
                "relate_set_cpals_graph": (I, [P, I]),
                "relate_footprint": (I, [P, I, I64, P, I, P]),
                "relate_release_cached_memory": (I, []),
                "relate_decode": (I, [P, P, P, P, P, P]),
                "relate_get_partitions": (I, [P, P, P, P]),
                "relate_gram": (I, [P, I64, I, I, P, P]),
                "relate_gram_noalloc": (I, [P, I64, I, I, P, P]),
                "relate_solve_rows": (I, [P, I64, I, I, P, P]),
                "relate_sync_status": (I, [P, P]),
                "relate_free": (None, [P]),
                "relate_status_string": (ctypes.c_char_p, [I]),
                "relate_last_error": (ctypes.c_char_p, []),
                "relate_version": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def relate_status_string(status: int) -> str:
    return lib().relate_status_string(int(status)).decode()


def relate_last_error() -> str:
    return lib().relate_last_error().decode()


def relate_version() -> str:
    return lib().relate_version().decode()


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise RelateError(rc, where)


def _ptr(x) -> int | None:
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


class Handle:
    """Owns a relate_handle_t; frees it on close()/garbage collection."""

    def __init__(self, raw: int, dims, nmodes: int):
        self._raw = ctypes.c_void_p(raw)
        self.dims = [int(d) for d in dims]
        self.nmodes = nmodes

    @property
    def raw(self):
        return self._raw

    def close(self):
        if self._raw and self._raw.value:
            lib().relate_free(self._raw)
            self._raw = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def relate_encode(coords, vals, dims, *, bit_order=None, partition_size: int = 0, conflict=None,
                  val_dtype=None, factor_dtype="f32", acc_dtype=None, stream=None,
                  smem_budget: int = 0, shard_rank: int = 0, shard_count: int = 1) -> Handle:
    """coords: (N, nnz) uint32 (torch CUDA tensor or host numpy), vals: (nnz,)
    f32/f64 of the same residency. Returns a Handle."""
    on_dev = _is_device(coords)
    if on_dev != _is_device(vals):
        raise ValueError("coords and vals must both be on the device or both on the host")
    if not on_dev:
        coords = np.ascontiguousarray(coords, dtype=np.uint32)
        vals = np.ascontiguousarray(vals)
    N = int(coords.shape[0])
    nnz = int(coords.shape[1]) if coords.ndim == 2 else 0
    vdt = str(vals.dtype)
    if val_dtype is None:
        val_dtype = "f64" if "float64" in vdt else "f32"
    fdt = _DTYPES[factor_dtype]
    adt = _DTYPES[acc_dtype] if acc_dtype is not None else (RELATE_F64 if fdt == RELATE_F64 else RELATE_F32)
    p = Params()
    lib().relate_params_default(ctypes.byref(p))
    order_buf = None
    if bit_order is not None:
        order_buf = np.ascontiguousarray(bit_order, dtype=np.int8)
        p.bit_order = order_buf.ctypes.data
        p.bit_order_len = int(order_buf.shape[0])
    p.partition_size = int(partition_size)
    if conflict is not None:
        for m, c in enumerate(conflict):
            p.conflict[m] = int(c)
    p.val_dtype = _DTYPES[val_dtype]
    p.factor_dtype = fdt
    p.acc_dtype = adt
    p.coords_on_device = 1 if on_dev else 0
    p.stream = _stream(stream)
    p.smem_budget = int(smem_budget)
    p.shard_rank = int(shard_rank)
    p.shard_count = int(shard_count)
    dims_arr = np.ascontiguousarray(dims, dtype=np.uint64)
    out = ctypes.c_void_p(0)
    rc = lib().relate_encode(_ptr(coords), _ptr(vals), dims_arr.ctypes.data, N, nnz, ctypes.byref(p),
                             ctypes.byref(out))
    _check(rc, "relate_encode")
    return Handle(out.value, dims_arr.tolist(), N)


def _ptr_array(tensors, n):
    arr = (ctypes.c_void_p * n)()
    for k in range(n):
        t = tensors[k] if k < len(tensors) else None
        arr[k] = _ptr(t) if t is not None else None
    return arr


def relate_mttkrp(h: Handle, mode: int, factors, R: int, out, stream=None) -> None:
    _check(lib().relate_mttkrp(h.raw, int(mode), _ptr_array(factors, h.nmodes), int(R), _ptr(out),
                               _stream(stream)), "relate_mttkrp")


def relate_cpals(h: Handle, R: int, iters: int, tol: float, factors, lam=None):
    """Runs CP-ALS in place on `factors` (device tensors). `lam`: optional
    output for lambda (R float64, a host numpy array or a CUDA tensor); a
    host array is made if None. Returns dict(lam, fit, iters, status,
    ridge_retries, fit_trace)."""
    if lam is None:
        lam = np.zeros(R, dtype=np.float64)
    trace = np.zeros(max(iters, 1), dtype=np.float64)
    info = CpalsInfo()
    info.fit_trace = trace.ctypes.data
    rc = lib().relate_cpals(h.raw, int(R), int(iters), float(tol), _ptr_array(factors, h.nmodes),
                            _ptr(lam), ctypes.byref(info))
    _check(rc, "relate_cpals")
    return {"lam": lam, "fit": info.fit, "iters": info.iters, "status": info.status,
            "ridge_retries": info.ridge_retries, "fit_trace": trace[:info.iters].copy()}


class MttkrpItem(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("mode", ctypes.c_int), ("factors", ctypes.c_void_p), ("R", ctypes.c_int),
                ("out", ctypes.c_void_p)]


def relate_mttkrp_batch(items, stream=None) -> None:
    """items: list of (handle, mode, factors, R, out); one persistent launch
    per group of compatible items (relate_mttkrp_batch)."""
    keep = []
    arr = (MttkrpItem * max(len(items), 1))()
    for i, (h, mode, factors, R, out) in enumerate(items):
        fp = _ptr_array(factors, h.nmodes)
        keep.append(fp)
        arr[i] = MttkrpItem(h.raw.value, int(mode), ctypes.cast(fp, ctypes.c_void_p), int(R), _ptr(out))
    _check(lib().relate_mttkrp_batch(arr, len(items), _stream(stream)), "relate_mttkrp_batch")


def relate_cpals_batch(handles, R, iters: int, tol: float, factors, stream, prev_fit=None):
    """CP-ALS of several problems in lockstep (relate_cpals_batch). handles: n
    Handles; R: n ranks; factors: n lists of device tensors (updated in place);
    stream: a non-default torch stream. Returns (n result dicts as
    relate_cpals's, status of the call)."""
    n = len(handles)
    hs = (ctypes.c_void_p * max(n, 1))(*[h.raw.value for h in handles])
    Rs = (ctypes.c_int * max(n, 1))(*[int(r) for r in R])
    fps = [_ptr_array(f, h.nmodes) for f, h in zip(factors, handles)]
    fp_arr = (ctypes.c_void_p * max(n, 1))(*[ctypes.cast(x, ctypes.c_void_p).value for x in fps])
    lams = [np.zeros(int(r), dtype=np.float64) for r in R]
    lam_arr = (ctypes.c_void_p * max(n, 1))(*[x.ctypes.data for x in lams])
    traces = [np.zeros(max(iters, 1), dtype=np.float64) for _ in range(n)]
    infos = (CpalsInfo * max(n, 1))()
    for i in range(n):
        infos[i].fit_trace = traces[i].ctypes.data
    pf = None
    if prev_fit is not None:
        pf = np.ascontiguousarray(prev_fit, dtype=np.float64)
    rc = lib().relate_cpals_batch(hs, n, Rs, int(iters), float(tol), fp_arr, lam_arr,
                                  pf.ctypes.data if pf is not None else None, infos, _stream(stream))
    out = []
    for i in range(n):
        it = infos[i].iters
        out.append({"lam": lams[i], "fit": infos[i].fit, "iters": it, "status": infos[i].status,
                    "ridge_retries": infos[i].ridge_retries, "fit_trace": traces[i][:it].copy()})
    if rc not in (0, -6, -7):  # NOT_PD / TIMEOUT are per problem (their status)
        _check(rc, "relate_cpals_batch")
    return out, rc


def relate_get_stats(h: Handle) -> dict:
    s = Stats()
    _check(lib().relate_get_stats(h.raw, ctypes.byref(s)), "relate_get_stats")
    N = s.nmodes
    return {"nmodes": N, "lp": s.lp, "key_bytes": s.key_bytes, "nnz": s.nnz,
            "partition_size": s.partition_size, "partitions": s.partitions,
            "dims": list(s.dims[:N]), "lbits": list(s.lbits[:N]), "field_offset": list(s.field_offset[:N]),
            "runs": list(s.runs[:N]), "distinct": list(s.distinct[:N]), "maxcount": list(s.maxcount[:N]),
            "bit_order": list(s.bit_order[:s.lp]), "nnz_total": s.nnz_total, "shard_lo": s.shard_lo}


def relate_get_conflict(h: Handle, mode: int, R: int) -> int:
    c = ctypes.c_int(0)
    _check(lib().relate_get_conflict(h.raw, int(mode), int(R), ctypes.byref(c)), "relate_get_conflict")
    return c.value


def relate_set_conflict(h: Handle, mode: int, c: int) -> None:
    _check(lib().relate_set_conflict(h.raw, int(mode), int(c)), "relate_set_conflict")


def relate_set_mode_plan(h: Handle, mode: int, depth: int = -1, level=None, col_passes: int = 0) -> None:
    """Fiber-factoring plan of one mode (depth -1 / level None / col_passes 0 = AUTO)."""
    buf = None
    if level is not None:
        buf = np.ascontiguousarray(level, dtype=np.int8)
    _check(lib().relate_set_mode_plan(h.raw, int(mode), int(depth), buf.ctypes.data if buf is not None else None,
                                      int(col_passes)), "relate_set_mode_plan")


def relate_get_mode_plan(h: Handle, mode: int, R: int) -> dict:
    d, p = ctypes.c_int(0), ctypes.c_int(0)
    lv = np.zeros(MAX_MODES, dtype=np.int8)
    _check(lib().relate_get_mode_plan(h.raw, int(mode), int(R), ctypes.byref(d), lv.ctypes.data, ctypes.byref(p)),
           "relate_get_mode_plan")
    return {"depth": d.value, "level": [int(x) for x in lv[:h.nmodes - 1]], "col_passes": p.value}


def relate_set_mode_kr(h: Handle, mode: int, kr: int = -1) -> None:
    """Khatri-Rao pair of one mode's factored MTTKRP (-1 AUTO, 0 off, 1 on)."""
    _check(lib().relate_set_mode_kr(h.raw, int(mode), int(kr)), "relate_set_mode_kr")


def relate_get_mode_kr(h: Handle, mode: int, R: int) -> dict:
    k, rows = ctypes.c_int(0), ctypes.c_uint64(0)
    _check(lib().relate_get_mode_kr(h.raw, int(mode), int(R), ctypes.byref(k), ctypes.byref(rows)),
           "relate_get_mode_kr")
    return {"kr": k.value, "rows": rows.value}


def relate_set_precision(h: Handle, factor_dtype, acc_dtype=None) -> None:
    fdt = _DTYPES[factor_dtype]
    adt = _DTYPES[acc_dtype] if acc_dtype is not None else (RELATE_F64 if fdt == RELATE_F64 else RELATE_F32)
    _check(lib().relate_set_precision(h.raw, fdt, adt), "relate_set_precision")


def relate_set_stream(h: Handle, stream) -> None:
    _check(lib().relate_set_stream(h.raw, _stream(stream)), "relate_set_stream")


REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p)


def relate_shard_range(nnz: int, rank: int, count: int) -> tuple[int, int]:
    lo, hi = ctypes.c_int64(0), ctypes.c_int64(0)
    lib().relate_shard_range(int(nnz), int(rank), int(count), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def relate_set_reduce_hook(h: Handle, fn) -> None:
    """fn(buf_ptr, count, dtype, stream_ptr) -> int: the all-reduce of a
    sharded CP-ALS (None removes it). The ctypes callback is kept on the
    handle for as long as it is set."""
    if fn is None:
        h._reduce_cb = None
        _check(lib().relate_set_reduce_hook(h.raw, None, None), "relate_set_reduce_hook")
        return

    def trampoline(buf, count, dtype, stream, user):
        try:
            return int(fn(buf, count, dtype, stream) or 0)
        except Exception:  # reported to the library as a failed reduction
            import traceback
            traceback.print_exc()
            return -1

    cb = REDUCE_FN(trampoline)
    h._reduce_cb = cb
    _check(lib().relate_set_reduce_hook(h.raw, ctypes.cast(cb, ctypes.c_void_p), None), "relate_set_reduce_hook")


class Footprint(ctypes.Structure):
    _fields_ = [("encode_peak", ctypes.c_uint64), ("resident", ctypes.c_uint64),
                ("cpals_workspace", ctypes.c_uint64), ("factors", ctypes.c_uint64)]


def relate_footprint(dims, nnz: int, R: int, factor_dtype="f32", val_dtype="f32", partition_size: int = 0,
                     coords_on_device: bool = False) -> dict:
    """Device bytes relate_encode / relate_cpals request for this shape (host
    only). 'peak' = max(encode_peak, resident + cpals_workspace) + factors."""
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.uint64))
    p = Params()
    lib().relate_params_default(ctypes.byref(p))
    p.partition_size = int(partition_size)
    p.val_dtype = _DTYPES[val_dtype]
    p.factor_dtype = _DTYPES[factor_dtype]
    p.acc_dtype = RELATE_F64 if factor_dtype == "f64" else RELATE_F32
    p.coords_on_device = int(bool(coords_on_device))
    f = Footprint()
    _check(lib().relate_footprint(d.ctypes.data, len(d), int(nnz), ctypes.byref(p), int(R), ctypes.byref(f)),
           "relate_footprint")
    out = {k: int(getattr(f, k)) for k, _ in Footprint._fields_}
    out["peak"] = max(out["encode_peak"], out["resident"] + out["cpals_workspace"]) + out["factors"]
    return out


def relate_release_cached_memory() -> None:
    """Trims the library's device-memory pool of the current device."""
    _check(lib().relate_release_cached_memory(), "relate_release_cached_memory")


def relate_set_cpals_graph(h: Handle, enable: bool) -> None:
    _check(lib().relate_set_cpals_graph(h.raw, int(bool(enable))), "relate_set_cpals_graph")


def relate_decode(h: Handle, coords_out=None, vals_out=None, perm_out=None, keys_out=None, stream=None) -> None:
    _check(lib().relate_decode(h.raw, _ptr(coords_out), _ptr(vals_out), _ptr(perm_out), _ptr(keys_out),
                               _stream(stream)), "relate_decode")


def relate_get_partitions(h: Handle, lo, hi, stream=None) -> None:
    _check(lib().relate_get_partitions(h.raw, _ptr(lo), _ptr(hi), _stream(stream)), "relate_get_partitions")


def relate_gram(A, R: int, dtype, G, stream=None) -> None:
    I = int(A.shape[0]) if A is not None else 0
    _check(lib().relate_gram(_ptr(A), I, int(R), _DTYPES[dtype], _ptr(G), _stream(stream)), "relate_gram")


def relate_solve_rows(M, R: int, dtype, W, stream=None) -> None:
    """In place M <- M W (the CP-ALS row update with W = V^{-1}); M (I x R)
    F64 or F32 on the device, W (R x R) FP64 on the device."""
    I = int(M.shape[0]) if M is not None else 0
    _check(lib().relate_solve_rows(_ptr(M), I, int(R), _DTYPES[dtype], _ptr(W), _stream(stream)), "relate_solve_rows")


def relate_sync_status(h: Handle, stream=None) -> None:
    _check(lib().relate_sync_status(h.raw, _stream(stream)), "relate_sync_status")


def relate_gram_noalloc(A, R: int, dtype, G, stream=None) -> None:
    """Gram step with the library's fixed scratch (no device allocation)."""
    I = int(A.shape[0]) if A is not None else 0
    _check(lib().relate_gram_noalloc(_ptr(A), I, int(R), _DTYPES[dtype], _ptr(G), _stream(stream)),
           "relate_gram_noalloc")


def relate_free(h: Handle) -> None:
    h.close()
