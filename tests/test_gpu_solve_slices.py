"""The FP64 row update M <- M W of CP-ALS on the tensor cores (relate_solve_rows:
exact integer slices of every row of M on its own scale and every column of W
on its own, exact slice products, 128-bit dot products rounded once).

Inputs are k * 2^e with integers k of at most 26 significant bits, the
scale spread over rows of M (31 binades) and over columns of W, so every
product M_ir W_rs is exact in FP64 and math.fsum of the products is the
correctly rounded reference. The bound is the slicing's: each entry keeps
55 bits below its row's (M) or column's (W) largest exponent, so
|D_is - ref| <= 2^-53 R max_r |M_ir| max_r |W_rs| + one rounding of ref.
"""
import math

import numpy as np
import pytest
import torch

import paper_2509_00280_gb300 as rl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _inputs(I, R, seed):
    rng = np.random.default_rng(seed)
    M = np.ldexp(rng.integers(-(2 ** 25), 2 ** 25, (I, R)).astype(np.float64), rng.integers(-30, 1, (I, 1)))
    W = np.ldexp(rng.integers(-(2 ** 25), 2 ** 25, (R, R)).astype(np.float64), rng.integers(-8, 9, (1, R)))
    return M, W


def _exact(M, W):
    I, R = M.shape
    out = np.empty((I, R))
    for i in range(I):
        for s in range(R):
            out[i, s] = math.fsum(M[i] * W[:, s])
    return out


def _gpu(M, W, dt="f64"):
    tdt = torch.float64 if dt == "f64" else torch.float32
    m = torch.from_numpy(M).to(DEV).to(tdt).contiguous()
    w = torch.from_numpy(W).to(DEV).contiguous()
    rl.relate_solve_rows(m, M.shape[1], dt, w)
    torch.cuda.synchronize()
    return m.double().cpu().numpy()


@pytest.mark.parametrize("I,R", [(1, 1), (127, 13), (128, 32), (129, 33), (300, 64), (2000, 64), (1000, 16)])
def test_fp64_row_update_within_the_slicing_bound(I, R):
    M, W = _inputs(I, R, seed=I * 7 + R)
    ref = _exact(M, W)
    D = _gpu(M, W)
    bound = 2.0 ** -52 * R * np.outer(np.abs(M).max(axis=1), np.abs(W).max(axis=0)) + np.spacing(np.abs(ref))
    assert np.isfinite(D).all()
    assert np.all(np.abs(D - ref) <= bound), (I, R, np.max(np.abs(D - ref) / bound))


def test_fp64_row_update_matches_float64_matmul_closely():
    """Well-scaled random inputs (no heavy tails): the sliced product is as
    close to the exact one as numpy's FP64 matmul is."""
    rng = np.random.default_rng(3)
    M, W = rng.standard_normal((5000, 64)), rng.standard_normal((64, 64))
    D = _gpu(M, W)
    ref = M @ W
    assert np.max(np.abs(D - ref)) <= 64 * 2.0 ** -52 * np.max(np.abs(M) @ np.abs(W))


def test_fp64_row_update_special_rows():
    M, W = _inputs(300, 24, seed=11)
    M[5] = 0.0
    M[7, 3] = np.nan
    D = _gpu(M, W)
    assert np.all(D[5] == 0.0)
    assert np.isnan(D[7]).all()
    ok = [i for i in range(300) if i not in (5, 7)]
    ref = _exact(M[ok], W)
    assert np.allclose(D[ok], ref, rtol=1e-13, atol=0)


def test_fp32_row_update():
    rng = np.random.default_rng(5)
    M, W = rng.standard_normal((3000, 48)), rng.standard_normal((48, 48))
    D = _gpu(M, W, "f32")
    ref = M.astype(np.float32).astype(np.float64) @ W.astype(np.float32).astype(np.float64)
    assert np.max(np.abs(D - ref)) <= 1e-5 * np.max(np.abs(ref))
