"""Parity at the full workload sizes, in the launch configuration the benchmark
times (default partition size, AUTO conflict strategy, the workload's rank and
factor precision).

The oracle cannot run a whole 50M-150M-nonzero MTTKRP in test time, so two
checks stand in for it:

* Masked values. The tensor keeps all its nonzeros (so the encoding, the
  partitions, the per-mode statistics, the conflict strategy and the tiles
  are those of the full workload) but only a random ~3M of them keep their
  value; the others are set to 0. By linearity of the MTTKRP (Sec. 2.2,
  Fig. 2) in the values, every output row must equal the oracle's MTTKRP of
  just the kept nonzeros: all rows of all modes are compared.
* Sampled rows. With the real values, each mode's most populated rows and
  random populated rows are compared with the oracle's MTTKRP over exactly
  the nonzeros of those rows (at most ~4M nonzeros per mode).

Tolerances are those of the small cases (relative Frobenius error): FP64
<= 1e-12 (the 150M workload in the benchmark's FP64 form); FP32 <= 1e-5; BF16 <= 1e-5 against the oracle fed the BF16-rounded factors and
<= 2e-2 against the unrounded factors. For the 50M-nonzero workload the
first CP-ALS iteration is also compared with the oracle's FP64 iteration on
the whole tensor (fit within 1e-3).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, encode_dev, factors_dev, rel_fro

pytestmark = pytest.mark.gpu

KEEP = 3_000_000       # nonzeros that keep their value in the masked check
ROW_BUDGET = 4_000_000  # nonzeros the oracle sums for the sampled rows of a mode
N_HOT, N_RANDOM = 8, 56


def _mttkrp_rows(h, n, dfs, R, rows=None, fdt="f32"):
    out = torch.empty((h.dims[n], R), dtype=torch.float64 if fdt == "f64" else torch.float32, device=DEV)
    rl.relate_mttkrp(h, n, dfs, R, out)
    torch.cuda.synchronize()
    if rows is not None:
        out = out[torch.from_numpy(rows).to(DEV)]
    return out.cpu().numpy().astype(np.float64)


def _sample_rows(counts, rng):
    """Hot rows (most populated first) and random populated rows, within the
    oracle's nonzero budget."""
    order = np.argsort(-counts, kind="stable")
    rows, used = [], 0
    for r in order[:N_HOT]:
        if counts[r] and used + counts[r] <= ROW_BUDGET:
            rows.append(r)
            used += counts[r]
    populated = np.nonzero((counts > 0) & (counts <= ROW_BUDGET // (2 * N_RANDOM)))[0]
    if populated.size:
        rows += list(rng.choice(populated, size=min(N_RANDOM, populated.size), replace=False))
    return np.unique(np.array(rows, dtype=np.int64))


def _oracle_rows(c, v64, dims, n, rows, fs64):
    """The oracle's MTTKRP over the nonzeros of the sampled rows; the rows are
    relabelled 0..k-1 so that its output is k x R."""
    sel = np.isin(c[n], rows)
    cs = c[:, sel].copy()
    cs[n] = np.searchsorted(rows, cs[n]).astype(np.uint32)
    dims_s = list(dims)
    dims_s[n] = len(rows)
    fs_s = list(fs64)
    fs_s[n] = np.zeros((len(rows), fs64[n].shape[1]))
    return oracle.mttkrp(cs, v64[sel], dims_s, n, fs_s)


@pytest.mark.parametrize("name,fdt", [("zipf3d-200Kx200Kx5K-50M", "f32"), ("zipf4d-5Mx1Mx100Kx24-150M", "f64"),
                                      ("zipf4d-5Mx1Mx100Kx24-150M", "f32"), ("zipf5d-10Mx10Mx1Mx1Kx100-100M", "bf16")])
def test_full_size(name, fdt):
    w = synth.WORKLOADS[name]
    spec, R = w["spec"], w["R"]
    tol = 1e-12 if fdt == "f64" else 1e-5
    c, v = synth.make_tensor(spec)  # values keep their stored dtype, as in the benchmark
    N = len(spec.dims)
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float64 if fdt == "f64" else np.float32)
    fs_unr = [f.astype(np.float64) for f in fs]
    fs_rnd = [oracle.round_bf16(f).astype(np.float64) for f in fs] if fdt == "bf16" else fs_unr
    dfs = factors_dev(fs, fdt)
    rng = np.random.default_rng(7)

    # masked values: full-size launch, every row compared
    keep = rng.random(spec.nnz) < KEEP / spec.nnz
    vm = np.where(keep, v, v.dtype.type(0))
    h = encode_dev(c, vm, spec.dims, factor_dtype=fdt)
    st = rl.relate_get_stats(h)
    assert st["nnz"] == spec.nnz and st["partition_size"] == 4096
    ck, vk = c[:, keep], v[keep].astype(np.float64)
    for n in range(N):
        got = _mttkrp_rows(h, n, dfs, R, fdt=fdt)
        strat = rl.relate_get_conflict(h, n, R)
        ref = oracle.mttkrp(ck, vk, spec.dims, n, fs_rnd)
        assert rel_fro(got, ref) <= tol, ("masked", name, n, strat)
        if fdt == "bf16":
            assert rel_fro(got, oracle.mttkrp(ck, vk, spec.dims, n, fs_unr)) <= 2e-2, ("masked", name, n)
        del got, ref
    h.close()

    # real values: sampled rows
    v64 = v.astype(np.float64)
    h = encode_dev(c, v, spec.dims, factor_dtype=fdt)
    for n in range(N):
        rows = _sample_rows(np.bincount(c[n], minlength=spec.dims[n]), rng)
        if rows.size == 0:
            continue
        got = _mttkrp_rows(h, n, dfs, R, rows, fdt=fdt)
        assert rel_fro(got, _oracle_rows(c, v64, spec.dims, n, rows, fs_rnd)) <= tol, ("rows", name, n)
        if fdt == "bf16":
            assert rel_fro(got, _oracle_rows(c, v64, spec.dims, n, rows, fs_unr)) <= 2e-2, ("rows", name, n)
    h.close()


def test_full_size_first_cpals_iteration():
    w = synth.WORKLOADS["zipf3d-200Kx200Kx5K-50M"]
    spec, R, fdt = w["spec"], w["R"], w["factor_dtype"]
    c, v = synth.make_tensor(spec)
    init = synth.init_factors(spec.dims, R, seed=0)
    ref = oracle.cpals(c, v.astype(np.float64), spec.dims, R, 1, 0.0, init)
    h = encode_dev(c, v, spec.dims, factor_dtype=fdt)
    res = rl.relate_cpals(h, R, 1, 0.0, factors_dev(init, fdt))
    h.close()
    assert res["status"] == 0 and res["iters"] == 1
    assert abs(res["fit"] - ref["fit_trace"][0]) <= 1e-3, (res["fit"], ref["fit_trace"][0])
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-3)
