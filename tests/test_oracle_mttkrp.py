"""Pins for the oracle's MTTKRP (CPU only).

Checked against: the dense definition X_(n) times the explicit Khatri-Rao
product on tiny tensors (Sec. 2.1 matricization and KRP, Sec. 2.2 MTTKRP),
exact big-integer sums, the all-ones closed form, linearity, and the fact
that the mode's own factor never enters.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _random_sparse(dims, density, rng, int_vals=None):
    cells = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.uint32).T
    keep = rng.random(cells.shape[1]) < density
    c = np.ascontiguousarray(cells[:, keep])
    if int_vals:
        v = rng.integers(int_vals[0], int_vals[1] + 1, c.shape[1]).astype(np.float64)
    else:
        v = rng.random(c.shape[1]) + 0.01
    return c, v


def _dense(c, v, dims):
    X = np.zeros(dims)
    X[tuple(c.astype(np.int64))] = v
    return X


def _unfold(X, n):
    """Kolda-Bader mode-n matricization: column index j = sum_{k != n} i_k J_k,
    J_k = prod_{m < k, m != n} I_m (earlier modes vary fastest)."""
    N = X.ndim
    other = [k for k in range(N) if k != n]
    Xn = np.moveaxis(X, n, 0)
    # after moveaxis the remaining axes are in increasing mode order; Fortran
    # order makes the earliest of them vary fastest
    return Xn.reshape(X.shape[n], -1, order="F"), other


def _khatri_rao(mats):
    """Column-wise Kronecker product mats[0] (.) mats[1] (.) ... (Sec. 2.1)."""
    K = mats[0]
    for B in mats[1:]:
        K = np.einsum("ir,jr->ijr", K, B).reshape(-1, K.shape[1])
    return K


def _dense_mttkrp(X, factors, n):
    Xn, other = _unfold(X, n)
    # earlier modes vary fastest in the columns, so the KRP lists the last
    # mode first: A_{N-1} (.) ... (.) A_0 (skipping n)
    K = _khatri_rao([factors[k] for k in reversed(other)])
    return Xn @ K


@pytest.mark.parametrize("dims", [(8, 7, 6), (5, 4, 3, 2), (3, 9)])
def test_matches_dense_unfolding_times_krp(dims):
    rng = np.random.default_rng(10)
    c, v = _random_sparse(dims, 0.3, rng)
    R = 5
    fs = [rng.random((d, R)) - 0.3 for d in dims]
    X = _dense(c, v, dims)
    for n in range(len(dims)):
        got = oracle.mttkrp(c, v, dims, n, fs)
        ref = _dense_mttkrp(X, fs, n)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_integer_exact_bitwise():
    rng = np.random.default_rng(11)
    dims = (9, 8, 7, 3)
    c, v = _random_sparse(dims, 0.5, rng, int_vals=(1, 8))
    R = 6
    fs = [rng.integers(0, 5, (d, R)).astype(np.float64) for d in dims]
    for n in range(len(dims)):
        got = oracle.mttkrp(c, v, dims, n, fs)
        exact = {}
        for e in range(c.shape[1]):
            row = int(c[n, e])
            for r in range(R):
                t = int(v[e])
                for k in range(len(dims)):
                    if k != n:
                        t *= int(fs[k][c[k, e], r])
                exact[(row, r)] = exact.get((row, r), 0) + t
        ref = np.zeros_like(got)
        for (row, r), s in exact.items():
            ref[row, r] = s
        assert np.array_equal(got, ref)


def test_all_ones_factors_is_slice_sum():
    rng = np.random.default_rng(12)
    dims = (40, 30, 20)
    c = np.stack([rng.integers(0, d, 3000) for d in dims]).astype(np.uint32)
    v = rng.random(3000)
    fs = [np.ones((d, 4)) for d in dims]
    for n in range(3):
        got = oracle.mttkrp(c, v, dims, n, fs)
        slice_sum = np.bincount(c[n], weights=v, minlength=dims[n])
        for r in range(4):
            np.testing.assert_allclose(got[:, r], slice_sum, rtol=1e-13, atol=0)


def test_linearity_and_own_factor_unused():
    rng = np.random.default_rng(13)
    dims = (30, 25, 20)
    c = np.stack([rng.integers(0, d, 2000) for d in dims]).astype(np.uint32)
    v1, v2 = rng.random(2000), rng.random(2000) - 0.5
    R = 8
    fs = [rng.random((d, R)) for d in dims]
    for n in range(3):
        m1 = oracle.mttkrp(c, v1, dims, n, fs)
        m2 = oracle.mttkrp(c, v2, dims, n, fs)
        m12 = oracle.mttkrp(c, 2.5 * v1 - 3.0 * v2, dims, n, fs)
        np.testing.assert_allclose(m12, 2.5 * m1 - 3.0 * m2, rtol=1e-12, atol=1e-12)
        k = (n + 1) % 3
        fs2 = list(fs)
        fs2[k] = 2.0 * fs[k] + 0.0
        np.testing.assert_allclose(oracle.mttkrp(c, v1, dims, n, fs2), 2.0 * m1, rtol=1e-13, atol=0)
        fs3 = list(fs)
        fs3[n] = rng.random((dims[n], R))
        assert np.array_equal(oracle.mttkrp(c, v1, dims, n, fs3), m1)


def test_input_order_does_not_matter():
    rng = np.random.default_rng(14)
    dims = (50, 40, 30)
    c = np.stack([rng.integers(0, d, 5000) for d in dims]).astype(np.uint32)
    v = rng.random(5000)
    fs = [rng.random((d, 7)) for d in dims]
    p = rng.permutation(5000)
    for n in range(3):
        a = oracle.mttkrp(c, v, dims, n, fs)
        b = oracle.mttkrp(c[:, p], v[p], dims, n, fs)
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=1e-15)


def test_compensated_sum_beats_naive_on_long_rows():
    """One output row fed by many terms of mixed magnitude: the oracle's
    Neumaier sum equals math.fsum (exact rounding) to a few ulp."""
    import math
    rng = np.random.default_rng(15)
    nnz = 20000
    c = np.zeros((2, nnz), dtype=np.uint32)
    c[1] = rng.integers(0, 3, nnz)
    v = rng.standard_normal(nnz) * 10.0 ** rng.integers(-8, 8, nnz)
    fs = [np.ones((1, 1)), np.ones((3, 1))]
    got = oracle.mttkrp(c, v, (1, 3), 0, fs)[0, 0]
    exact = math.fsum(v.tolist())
    assert abs(got - exact) <= 4 * np.spacing(abs(exact)) + 1e-300


def test_openmp_baseline_mttkrp_matches_the_oracle():
    """The CPU baseline's OpenMP MTTKRP (private copies for a short mode,
    atomics for a long one) equals the compensated oracle up to rounding."""
    spec = synth.TensorSpec("omp4d", (3000, 800, 90, 24), 200_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="uniform", value_dtype="f64", seed=12)
    c, v = synth.make_tensor(spec)
    fs = synth.init_factors(spec.dims, 24, seed=1)
    for n in range(4):
        ref = oracle.mttkrp(c, v, spec.dims, n, fs)
        for limit in (0, 1 << 30):  # atomics / per-thread copies
            got = oracle.mttkrp_omp(c, v, spec.dims, n, fs, 4, priv_limit=limit)
            assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), (n, limit)
