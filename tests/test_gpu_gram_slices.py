"""The Gram on the tensor cores for FP64 inputs (exact integer slices of
every entry, exact BF16 products, exact FP32 integer sums per 128-row period)
and FP32 inputs (three BF16 terms per entry, FP32 accumulation per 128
rows, compensated FP32 sums across those periods).

Inputs are k * 2^e with integer k of at most 26 (FP64) or 24 (FP32)
significant bits and a per-row scale 2^e spread over 31 binades, so that the
columns are heavy-tailed (a few rows dominate every column, as in the factor
updates of a Zipf-distributed mode). Every product a_ir a_is is then exact in
FP64, and math.fsum of the products is the correctly rounded Gram: the
reference has no error of its own. The bounds, relative to
||A(:, r)|| ||A(:, s)||: FP64, the truncation of each entry 55 bits below its
column's largest exponent, 2^-53 sqrt(I) (with a factor 2 of slack); a
slicing that dropped the low-order pair products would be off by about
I * 2^-53 on these inputs and fail the larger cases. FP32, the dropped terms
of the three-term split (2^-22) plus FP32 summation over the rows of one
128-row period (worst case linear in them), plus the compensated sum of the
periods (two more units of 2^-24).
"""
import math

import numpy as np
import pytest
import torch

import paper_2509_00280_gb300 as rl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TORCH = {"f64": torch.float64, "f32": torch.float32}
BITS = {"f64": 26, "f32": 24}


def _bound(dt, I):
    if dt == "f64":
        return 2.0 * 2.0 ** -53 * math.sqrt(I)
    # rows one block sums plainly in FP32: the launch takes
    # min(152, ceil(I / 64)) blocks of ceil(I / blocks) rows, in periods of 128
    blocks = min(152, max(1, -(-I // 64)))
    return 2.0 ** -22 + (min(-(-I // blocks), 128) + 2) * 2.0 ** -24


def _norm_err(G, ref):
    norms = np.sqrt(np.diag(ref))
    return np.abs(G - ref) / np.maximum(np.outer(norms, norms), 1e-300)


def _heavy(I, R, dt, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(-(2 ** (BITS[dt] - 1)), 2 ** (BITS[dt] - 1), (I, R)).astype(np.float64)
    e = rng.integers(-30, 1, (I, 1))
    return np.ldexp(k, e)


def _exact_gram(A):
    R = A.shape[1]
    G = np.empty((R, R))
    for r in range(R):
        for s in range(r, R):
            G[r, s] = G[s, r] = math.fsum(A[:, r] * A[:, s])
    return G


def _gpu_gram(A, dt, offset=0):
    I, R = A.shape
    flat = torch.zeros(I * R + offset, dtype=TORCH[dt], device=DEV)
    flat[offset:] = torch.from_numpy(A.reshape(-1)).to(DEV).to(TORCH[dt])
    t = flat[offset:].view(I, R)  # offset 1: a view 8 (or 4) bytes past a 16-byte boundary
    G = torch.full((R, R), float("nan"), dtype=torch.float64, device=DEV)
    rl.relate_gram(t, R, dt, G)
    torch.cuda.synchronize()
    return G.cpu().numpy()


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("I,R", [(1, 1), (63, 13), (64, 32), (65, 33), (129, 64), (1000, 8), (20011, 64)])
def test_sliced_gram_within_the_slicing_bound(dt, I, R):
    A = _heavy(I, R, dt, seed=I * 100 + R)
    ref = _exact_gram(A)
    G = _gpu_gram(A, dt, offset=1 if I % 2 else 0)
    err = _norm_err(G, ref)
    assert np.isfinite(G).all()
    assert err.max() <= _bound(dt, I), (dt, I, R, err.max())


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_sliced_gram_zero_and_nonfinite_columns(dt):
    A = _heavy(3000, 16, dt, seed=5)
    A[:, 3] = 0.0
    G = _gpu_gram(A, dt)
    assert np.all(G[3, :] == 0.0) and np.all(G[:, 3] == 0.0)
    ok = [c for c in range(16) if c != 3]
    ref = _exact_gram(A)
    assert _norm_err(G[np.ix_(ok, ok)], ref[np.ix_(ok, ok)]).max() <= _bound(dt, 3000)
    A[17, 5] = np.inf
    G = _gpu_gram(A, dt)
    assert np.isnan(G[5, :]).all() and np.isnan(G[:, 5]).all()
    assert np.isfinite(G[np.ix_([0, 1], [0, 1])]).all()


def test_sliced_gram_is_deterministic():
    A = _heavy(50_000, 64, "f64", seed=9)
    a = _gpu_gram(A, "f64")
    b = _gpu_gram(A, "f64")
    assert np.array_equal(a, b)
