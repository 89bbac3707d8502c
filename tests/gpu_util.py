"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

import paper_2509_00280_gb300 as rl

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_fro(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def encode_dev(coords, vals, dims, **kw):
    return rl.relate_encode(to_dev(coords), to_dev(vals), dims, **kw)


def decode_all(h, nnz, N, val_dtype):
    c = torch.empty((N, nnz), dtype=torch.int32, device=DEV)
    v = torch.empty(nnz, dtype=torch.float64 if val_dtype == "f64" else torch.float32, device=DEV)
    p = torch.empty(nnz, dtype=torch.int32, device=DEV)
    k = torch.empty((nnz, 2), dtype=torch.int64, device=DEV)
    rl.relate_decode(h, c, v, p, k)
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32)
    keys = k.cpu().numpy().view(np.uint64)
    return u32(c), v.cpu().numpy(), u32(p), keys[:, 0].copy(), keys[:, 1].copy()


def factors_dev(fs, dtype):
    return [torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64)).to(DEV).to(TORCH_DT[dtype]).contiguous()
            for f in fs]


def mttkrp_dev(h, mode, dfs, R, acc="f32"):
    out = torch.empty((h.dims[mode], R), dtype=torch.float64 if acc == "f64" else torch.float32, device=DEV)
    rl.relate_mttkrp(h, mode, dfs, R, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)
