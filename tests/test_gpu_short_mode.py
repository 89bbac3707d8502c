"""The AUTO rule's short modes (Sec. 4.1.3: the synchronisation follows the
fiber statistics), against the CPU oracle.

A 4-mode tensor of 1M nonzeros whose 24-row mode puts about 41K nonzeros on
every row: AUTO takes SEGMENTED with every row of that mode in the per-block
copy (its output is at most 16 KB). Checked for FP64, FP32 and BF16 factors, with 16-byte
aligned factors (vector path) and with factors one element off 16 bytes
(scalar path: no per-block copies, every run flushed by global atomics).
Tolerances as for every MTTKRP test: FP64 1e-12, FP32 1e-5, BF16 1e-5
against the oracle fed the BF16-rounded factors.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, TORCH_DT, encode_dev, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module")
def short_mode_tensor():
    spec = synth.TensorSpec("short-mode-4d", (3000, 2000, 500, 24), 1_000_000,
                            (("zipf", 1.1),) * 3 + (("uniform",),), values="uniform", value_dtype="f32", seed=41)
    c, v = synth.make_tensor(spec)
    return spec, c, v


def _factors(dims, R, dtype, offset):
    """Factors on the device; offset = 1 shifts each start by one element."""
    fs = synth.init_factors(dims, R, seed=5)
    if dtype == "bf16":
        fs = [oracle.round_bf16(f.astype(np.float32)).astype(np.float64) for f in fs]
    out = []
    for f in fs:
        flat = torch.zeros(f.size + offset, dtype=TORCH_DT[dtype], device=DEV)
        view = flat[offset:].view(f.shape)
        view.copy_(torch.from_numpy(f).to(DEV).to(TORCH_DT[dtype]))
        out.append(view)
    return fs, out


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("fdt", ["f64", "f32", "bf16"])
def test_short_hot_mode_auto_segmented(short_mode_tensor, fdt, offset):
    spec, c, v = short_mode_tensor
    R = 32
    h = encode_dev(c, v.astype(np.float64) if fdt == "f64" else v, spec.dims, factor_dtype=fdt)
    st = rl.relate_get_stats(h)
    assert st["maxcount"][3] >= 2 ** 15 and st["dims"][3] == 24
    assert rl.relate_get_conflict(h, 3, R) == rl.RELATE_CONFLICT_SEGMENTED
    fs, dfs = _factors(spec.dims, R, fdt, offset)
    if offset:
        assert all(t.data_ptr() % 16 != 0 for t in dfs)
    acc = torch.float64 if fdt == "f64" else torch.float32
    for n in (3, 0):
        out = torch.empty((spec.dims[n], R), dtype=acc, device=DEV)
        rl.relate_mttkrp(h, n, dfs, R, out)
        torch.cuda.synchronize()
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
        assert rel_fro(out.cpu().numpy(), ref) <= TOL[fdt], (fdt, offset, n)
    rl.relate_sync_status(h)
    h.close()


def test_hundred_row_mode_keeps_every_row_in_the_block_copy():
    """A 100-row mode of a 5-mode BF16 tensor (6.4 KB of FP32 output at R = 16,
    ~10K nonzeros per row): AUTO SEGMENTED with all rows in the per-block
    copy, within the BF16 tolerance (1e-5 against the rounded factors)."""
    spec = synth.TensorSpec("short5d", (4000, 3000, 500, 60, 100), 1_000_000, (("zipf", 1.3),) * 2 + (("uniform",),) * 3,
                            values="uniform", value_dtype="f32", seed=42)
    c, v = synth.make_tensor(spec)
    R = 16
    h = encode_dev(c, v, spec.dims, factor_dtype="bf16")
    assert rl.relate_get_conflict(h, 4, R) == rl.RELATE_CONFLICT_SEGMENTED
    fs, dfs = _factors(spec.dims, R, "bf16", 0)
    for n in (4, 3):
        out = torch.empty((spec.dims[n], R), dtype=torch.float32, device=DEV)
        rl.relate_mttkrp(h, n, dfs, R, out)
        torch.cuda.synchronize()
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
        assert rel_fro(out.cpu().numpy(), ref) <= 1e-5, n
    h.close()
