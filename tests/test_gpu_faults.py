"""Failure detection without a GPU fault.

RELATE_FAULT is the library's host-side test hook:
* "alloc": every library allocation fails as if the device were out of
  memory; relate_encode must return RELATE_ERR_OOM, leave no handle, and the
  next call (hook unset) must work.
* "timeout": every MTTKRP launch skips its first tile copy and waits on it
  with a ~50 ms limit; the bounded wait runs out, the kernel sets the
  handle's error flag and returns, and the host reads RELATE_ERR_TIMEOUT
  (relate_sync_status, relate_cpals). No trap, no fault: the context stays
  usable and the next MTTKRP (hook unset) matches the oracle.
* "gram_timeout": the tensor-core Gram (BF16 inputs directly, FP32 / FP64
  inputs as integer slices) issues no MMA and waits for their completion
  with the same short limit; relate_gram and
  relate_cpals report RELATE_ERR_TIMEOUT, and with the hook unset the same
  calls succeed.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import encode_dev, factors_dev, mttkrp_dev, rel_fro

pytestmark = pytest.mark.gpu

OOM, TIMEOUT = -5, -7


def _small():
    spec = synth.scaled(synth.WORKLOADS["zipf3d-200Kx200Kx5K-50M"]["spec"], 100_000, dims=(5000, 4000, 300))
    c, v = synth.make_tensor(spec)
    return spec, c, v


def test_injected_allocation_failure(monkeypatch):
    spec, c, v = _small()
    monkeypatch.setenv("RELATE_FAULT", "alloc")
    with pytest.raises(rl.RelateError) as ei:
        encode_dev(c, v, spec.dims)
    assert ei.value.status == OOM
    monkeypatch.delenv("RELATE_FAULT")
    h = encode_dev(c, v, spec.dims)
    assert rl.relate_get_stats(h)["nnz"] == spec.nnz
    h.close()


def test_injected_timeout_is_reported_and_the_context_stays_usable(monkeypatch):
    spec, c, v = _small()
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float32)
    h = encode_dev(c, v, spec.dims, factor_dtype="f32")
    dfs = factors_dev(fs, "f32")
    out = torch.empty((spec.dims[0], R), dtype=torch.float32, device="cuda")
    monkeypatch.setenv("RELATE_FAULT", "timeout")
    rl.relate_mttkrp(h, 0, dfs, R, out)  # launches; the kernel gives up its wait
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_sync_status(h)
    assert ei.value.status == TIMEOUT
    rl.relate_sync_status(h)  # the flag was cleared by the read
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_cpals(h, R, 2, 0.0, factors_dev(fs, "f32"))
    assert ei.value.status == TIMEOUT
    monkeypatch.delenv("RELATE_FAULT")
    rl.relate_sync_status(h)
    ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, 0, [f.astype(np.float64) for f in fs])
    assert rel_fro(mttkrp_dev(h, 0, dfs, R), ref) <= 1e-5
    h.close()


@pytest.mark.parametrize("dt", ["bf16", "f32", "f64"])
def test_injected_tensor_core_gram_timeout_is_reported(monkeypatch, dt):
    rng = np.random.default_rng(31)
    A = factors_dev([rng.random((20000, 32))], dt)[0]
    G = torch.empty((32, 32), dtype=torch.float64, device="cuda")
    monkeypatch.setenv("RELATE_FAULT", "gram_timeout")
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_gram(A, 32, dt, G)
    assert ei.value.status == TIMEOUT
    spec, c, v = _small()
    fs = synth.init_factors(spec.dims, 16, seed=0, dtype=np.float32)
    h = encode_dev(c, v, spec.dims, factor_dtype=dt)
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_cpals(h, 16, 2, 0.0, factors_dev(fs, dt))
    assert ei.value.status == TIMEOUT
    monkeypatch.delenv("RELATE_FAULT")
    rl.relate_gram(A, 32, dt, G)
    torch.cuda.synchronize()
    exact = A.to(torch.float64).T @ A.to(torch.float64)
    assert float(torch.linalg.norm(G - exact) / torch.linalg.norm(exact)) <= (1e-13 if dt == "f64" else 2e-5)
    res = rl.relate_cpals(h, 16, 2, 0.0, factors_dev(fs, dt))
    assert res["status"] == 0 and np.isfinite(res["fit"])
    h.close()
