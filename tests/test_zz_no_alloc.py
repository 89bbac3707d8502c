"""relate_gram_noalloc against relate_gram.

relate_gram_noalloc serves callers that cannot allocate device memory when
they compute a Gram matrix (an application whose device memory already
belongs to its own pool, or a loop that cannot afford an allocator call): its
partial sums live in a fixed array inside the library. This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import paper_2509_00280_gb300 as rl

pytestmark = pytest.mark.gpu

# FP32/BF16 inputs accumulate in FP32 over a block's rows; FP64 stays FP64
# (the same tolerances as the relate_gram test)
TOL = {"f64": 1e-13, "f32": 2e-5, "bf16": 2e-5}
TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_noalloc_gram_matches_relate_gram_twice_in_a_row(dtype):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(77)
    # two calls in a row with different shapes: the second must not see the
    # first call's partial sums in the shared array
    for I, R in ((200_000, 32), (7_777, 13)):
        A = torch.from_numpy(rng.random((I, R))).to(dev).to(TORCH[dtype]).contiguous()
        G_ref = torch.empty((R, R), dtype=torch.float64, device=dev)
        G = torch.full((R, R), float("nan"), dtype=torch.float64, device=dev)
        rl.relate_gram(A, R, dtype, G_ref)
        rl.relate_gram_noalloc(A, R, dtype, G)
        torch.cuda.synchronize()
        assert torch.isfinite(G).all()
        assert _rel(G, G_ref) <= TOL[dtype], (dtype, I, R)
        exact = A.to(torch.float64).T @ A.to(torch.float64)
        assert _rel(G, exact) <= TOL[dtype], (dtype, I, R)


def test_noalloc_gram_rejects_rank_beyond_the_fixed_scratch():
    dev = torch.device("cuda:0")
    A = torch.ones((10, 65), dtype=torch.float32, device=dev)
    G = torch.empty((65, 65), dtype=torch.float64, device=dev)
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_gram_noalloc(A, 65, "f32", G)
    assert ei.value.status == -1 and "[1, 64]" in str(ei.value)


def test_noalloc_gram_reports_a_tensor_core_timeout_and_recovers(monkeypatch):
    """The tensor-core path's bounded-wait status word lives in the shared
    array: a timed-out call (RELATE_FAULT=gram_timeout issues no MMA, so the
    waits run out) returns RELATE_ERR_TIMEOUT, and the next call, which
    clears the word first, succeeds and matches relate_gram."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(78)
    A = torch.from_numpy(rng.random((50_000, 64))).to(dev).to(torch.bfloat16).contiguous()
    G = torch.empty((64, 64), dtype=torch.float64, device=dev)
    monkeypatch.setenv("RELATE_FAULT", "gram_timeout")
    with pytest.raises(rl.RelateError) as ei:
        rl.relate_gram_noalloc(A, 64, "bf16", G)
    assert ei.value.status == -7
    monkeypatch.delenv("RELATE_FAULT")
    G_ref = torch.empty((64, 64), dtype=torch.float64, device=dev)
    rl.relate_gram(A, 64, "bf16", G_ref)
    rl.relate_gram_noalloc(A, 64, "bf16", G)
    torch.cuda.synchronize()
    assert torch.isfinite(G).all()
    assert _rel(G, G_ref) <= TOL["bf16"]
