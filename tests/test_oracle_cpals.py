"""Pins for the oracle's dense CP-ALS remainder (CPU only).

Checked against: numpy linear algebra for the Gram / Cholesky / solve
residuals, recovery of planted exact low-rank tensors, the fit formula
against the explicit dense residual, and the ALS monotonicity property.
"""
import numpy as np
import pytest
import torch

import oracle


def test_gram_cholesky_solve():
    rng = np.random.default_rng(20)
    A = rng.random((300, 12))
    G = oracle.gram(A)
    np.testing.assert_allclose(G, A.T @ A, rtol=1e-13)
    L = oracle.cholesky(G)
    assert np.allclose(np.triu(L, 1), 0)
    np.testing.assert_allclose(L @ L.T, G, rtol=1e-12, atol=1e-12 * np.abs(G).max())
    M = rng.standard_normal((50, 12))
    X = oracle.solve_rows(M, G)
    assert np.linalg.norm(X @ G - M) <= 1e-12 * np.linalg.norm(M) * np.linalg.cond(G) ** 0.5
    with pytest.raises(oracle.OracleError):
        oracle.cholesky(-np.eye(3))


def test_ridge_retry_on_a_singular_normal_matrix():
    """The Hadamard product of Grams is positive semidefinite; it is singular
    when a factor has a zero column or two equal columns, and then the first
    Cholesky meets a zero pivot. The retry factors V + 1e-12 tr(V)/R I.
    [[1,1],[1,1]] (B = [1 1], a repeated column): the second pivot is exactly
    1 - 1 = 0. The ridge's scale is pinned by L L^T against V + ridge I at
    1e-14, well below the ridge itself (1e-12); a ridge with the wrong sign
    fails again (NOT_PD)."""
    V = np.array([[1.0, 1.0], [1.0, 1.0]])
    with pytest.raises(oracle.OracleError):
        oracle.cholesky(V)
    L, ridged = oracle.factor_normal(V)
    assert ridged == 1
    W = V + 1e-12 * np.trace(V) / 2 * np.eye(2)
    assert np.abs(L @ L.T - W).max() <= 1e-14
    assert np.abs(np.diag(L @ L.T - V) - 1e-12).max() <= 1e-14
    # a V that factors at once takes no ridge
    L0, r0 = oracle.factor_normal(np.array([[4.0, 2.0], [2.0, 3.0]]))
    assert r0 == 0 and np.allclose(L0 @ L0.T, [[4.0, 2.0], [2.0, 3.0]], rtol=0, atol=1e-15)


def test_ridge_retry_with_a_zero_factor_column_solves_the_ridged_system():
    """A zero column r of a factor makes row and column r of V zero: the
    pivot of column r is exactly 0, the retry succeeds, and the solve gives
    A = M (V + ridge I)^{-1}; a right-hand side with a zero column r (the
    MTTKRP of that factor) keeps column r of A exactly zero."""
    rng = np.random.default_rng(27)
    B = rng.random((60, 6))
    B[:, 3] = 0.0
    C = rng.random((50, 6))
    V = (B.T @ B) * (C.T @ C)
    assert np.all(V[3] == 0.0) and np.all(V[:, 3] == 0.0)
    L, ridged = oracle.factor_normal(V)
    assert ridged == 1
    ridge = 1e-12 * np.trace(V) / 6
    W = V + ridge * np.eye(6)
    assert np.abs(L @ L.T - W).max() <= 1e-13 * np.abs(W).max()
    assert abs(L[3, 3] ** 2 - ridge) <= 1e-12 * ridge and np.all(L[3, :3] == 0.0)
    M = rng.standard_normal((40, 6))
    M[:, 3] = 0.0
    A = oracle.solve_rows(M, V)
    assert np.all(A[:, 3] == 0.0)
    assert np.linalg.norm(A @ W - M) <= 1e-12 * np.linalg.norm(M) * np.linalg.cond(W[np.ix_([0, 1, 2, 4, 5],
                                                                                             [0, 1, 2, 4, 5])])
    np.testing.assert_allclose(A, M @ np.linalg.inv(W), rtol=1e-9, atol=1e-12)


def test_cpals_with_a_zero_initial_column_takes_the_ridge_every_mode():
    """A zero column in one initial factor makes every mode's V singular in
    the first sweep (the zero column propagates): the oracle counts one ridge
    retry per mode and iteration, the zero column stays zero, and the other
    columns follow the run without it within the ridge's perturbation."""
    rng = np.random.default_rng(28)
    dims = (30, 25, 20)
    X = (rng.random(dims) < 0.2) * rng.random(dims)
    c, v = _to_coo(X)
    R, iters = 4, 3
    init = [rng.random((d, R)) for d in dims]
    init[2][:, 1] = 0.0
    res = oracle.cpals(c, v, dims, R, iters, 0.0, init)
    assert res["ridges"] == 3 * iters
    for f in res["factors"]:
        assert np.all(f[:, 1] == 0.0)
    assert res["lam"][1] == 0.0
    keep = [0, 2, 3]
    ref = oracle.cpals(c, v, dims, 3, iters, 0.0, [f[:, keep] for f in init])
    assert ref["ridges"] == 0
    assert np.max(np.abs(res["fit_trace"] - ref["fit_trace"])) <= 1e-9
    np.testing.assert_allclose(res["lam"][keep], ref["lam"], rtol=1e-8)


def _cp_dense(lam, fs):
    N = len(fs)
    letters = "abcdefgh"[:N]
    spec = ",".join(f"{l}r" for l in letters) + ",r->" + letters
    return np.einsum(spec, *fs, lam)


def _to_coo(X, thresh=0.0):
    idx = np.nonzero(np.abs(X) > thresh)
    c = np.stack(idx).astype(np.uint32)
    return c, X[idx]


def test_planted_dense_rank3_recovered():
    rng = np.random.default_rng(21)
    dims = (12, 10, 8)
    true = [rng.random((d, 3)) + 0.1 for d in dims]
    X = _cp_dense(np.array([3.0, 2.0, 1.0]), true)
    c, v = _to_coo(X)
    assert c.shape[1] == 12 * 10 * 8
    init = [rng.random((d, 3)) for d in dims]
    res = oracle.cpals(c, v, dims, 3, 1000, 0.0, init)  # collinear positive factors swamp slowly
    assert res["fit_trace"][-1] > 0.9999


def test_planted_block_disjoint_sparse_rankR_recovered():
    rng = np.random.default_rng(22)
    R = 4
    block = (5, 4, 3)
    dims = tuple(b * R for b in block)
    fs = [np.zeros((d, R)) for d in dims]
    for r in range(R):
        for k in range(3):
            fs[k][r * block[k]:(r + 1) * block[k], r] = rng.random(block[k]) + 0.5
    X = _cp_dense(np.ones(R), fs)
    c, v = _to_coo(X)
    assert c.shape[1] == R * 5 * 4 * 3
    # ALS has spurious local minima on this tensor from arbitrary starts, so
    # start from the planted factors blurred by dense positive noise: every
    # entry is perturbed and the block structure is hidden in the start
    init = [f + 0.25 * rng.random(f.shape) for f in fs]
    res = oracle.cpals(c, v, dims, R, 1000, 0.0, init)
    assert res["fit_trace"][-1] > 0.9999


def test_fit_formula_matches_explicit_residual_and_is_monotone():
    rng = np.random.default_rng(23)
    dims = (9, 7, 6, 4)
    X = (rng.random(dims) < 0.25) * rng.random(dims)
    c, v = _to_coo(X)
    R = 3
    init = [rng.random((d, R)) for d in dims]
    for iters in (1, 2, 5):
        res = oracle.cpals(c, v, dims, R, iters, 0.0, init)
        Xh = _cp_dense(res["lam"], res["factors"])
        explicit = 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
        assert abs(explicit - res["fit_trace"][-1]) <= 1e-12
        for f in res["factors"]:  # columns have unit 2-norm
            np.testing.assert_allclose(np.linalg.norm(f, axis=0), 1.0, rtol=1e-13)
    tr = oracle.cpals(c, v, dims, R, 30, 0.0, init)["fit_trace"]
    assert np.all(np.diff(tr) >= -1e-12)


def test_each_mode_update_solves_normal_equations():
    """After a one-iteration run on a 3-mode tensor, the last mode's factor
    (times lambda) solves A V = M with V the Hadamard product of the other
    two modes' Grams and M the MTTKRP with those (normalised) factors."""
    rng = np.random.default_rng(24)
    dims = (11, 9, 7)
    X = (rng.random(dims) < 0.3) * rng.random(dims)
    c, v = _to_coo(X)
    R = 4
    init = [rng.random((d, R)) for d in dims]
    res = oracle.cpals(c, v, dims, R, 1, 0.0, init)
    A0, A1, A2 = res["factors"]
    M = oracle.mttkrp(c, v, dims, 2, [A0, A1, A2])
    V = (A0.T @ A0) * (A1.T @ A1)
    Araw = A2 * res["lam"]
    assert np.linalg.norm(Araw @ V - M) <= 1e-12 * np.linalg.norm(M)


def test_stops_on_tolerance():
    rng = np.random.default_rng(25)
    dims = (12, 10, 8)
    true = [rng.random((d, 2)) + 0.1 for d in dims]
    c, v = _to_coo(_cp_dense(np.array([1.0, 0.5]), true))
    res = oracle.cpals(c, v, dims, 2, 500, 1e-6, [rng.random((d, 2)) for d in dims])
    assert res["iters"] < 500
    tr = res["fit_trace"]
    assert abs(tr[-1] - tr[-2]) < 1e-6 and (len(tr) < 3 or abs(tr[-2] - tr[-3]) >= 1e-6)


def test_round_bf16_rne():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3, 65504.0, 1.0 + 2 ** -7],
                 dtype=np.float32)
    got = oracle.round_bf16(x)
    assert got[0] == 1.0
    assert got[1] == 1.0                  # tie -> even (down)
    assert got[2] == np.float32(1.0 + 2 ** -6)  # tie -> even (up)
    assert got[6] == np.float32(1.0 + 2 ** -7)  # exactly representable
    rng = np.random.default_rng(26)
    y = (rng.standard_normal(100000) * 10.0 ** rng.integers(-20, 20, 100000)).astype(np.float32)
    ref = torch.from_numpy(y).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.round_bf16(y), ref)
