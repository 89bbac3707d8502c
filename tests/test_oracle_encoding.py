"""Pins for the oracle's encoding functions (CPU only).

Each test checks the oracle against something other than itself: the
paper's worked 4x8x2 example (Sec. 3.3.1, Fig. 5), the interleaving count of
Eq. 1, textbook special cases (row-major linear index, magic-number Morton
code) and pure-Python brute force on tiny inputs.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden


def _all_orders(lbits):
    base = [n for n, l in enumerate(lbits) for _ in range(l)]
    return sorted(set(itertools.permutations(base)))


def test_alto_worked_example():
    g = read_golden("alto_4x8x2.txt")
    dims = [int(x) for x in g["dims"]]
    lbits, lp = oracle.bit_budget(dims)
    assert lbits == [int(x) for x in g["lbits"]] and lp == int(g["lp"][0])
    order = oracle.alto_order(dims)
    pos0 = [t for t, n in enumerate(order) if n == 0]
    assert pos0 == [int(x) for x in g["mode0_bit_positions"]]
    # "starting with the shortest mode": b^0 is the 1-bit mode, the top bit
    # belongs to the longest mode (space split along the longest mode first)
    assert order[0] == 2 and order[-1] == 1
    assert oracle.check_order(dims, order)


def test_interleavings_of_worked_example():
    g = read_golden("alto_4x8x2.txt")
    dims = [int(x) for x in g["dims"]]
    lbits, lp = oracle.bit_budget(dims)
    orders = _all_orders(lbits)
    assert len(orders) == int(g["interleavings"][0])
    assert math.factorial(lp) == int(g["orderings_all_bits"][0])
    cells = np.array(list(itertools.product(range(4), range(8), range(2))), dtype=np.uint32).T
    for order in orders:
        assert oracle.check_order(dims, order)
        lo, hi = oracle.encode(cells, dims, order)
        assert not hi.any()
        # a bijection of the 64-cell box onto [0, 2^l(p)): storage is l(p)
        # bits whatever the order (Sec. 4.2: storage depends on shape only)
        assert sorted(lo.tolist()) == list(range(64))
        back = oracle.decode(lo, hi, dims, order)
        assert np.array_equal(back, cells)


@pytest.mark.parametrize("lbits", [(2, 2), (2, 1, 1), (1, 1, 1, 1), (3, 2), (2, 3, 1)])
def test_valid_orders_count_is_multinomial(lbits):
    """Brute force over all N^l(p) sequences: the oracle accepts exactly the
    multinomial number of Eq. 1."""
    dims = [2 ** l for l in lbits]
    N, lp = len(lbits), sum(lbits)
    accepted = sum(oracle.check_order(dims, seq) for seq in itertools.product(range(N), repeat=lp))
    expect = math.factorial(lp)
    for l in lbits:
        expect //= math.factorial(l)
    assert accepted == expect


def test_search_space_counts_printed_in_paper():
    g = read_golden("search_space_counts.txt")
    tol = float(g["rel_tol"][0])
    allf = math.factorial(32)
    inter = math.factorial(32) // math.factorial(8) ** 4
    assert abs(allf / float(g["all_formats_4x8"][0]) - 1) < tol
    assert abs(inter / float(g["interleaved_4x8"][0]) - 1) < tol
    # the brute-force multinomial count above and this closed form agree
    assert inter == math.comb(32, 8) * math.comb(24, 8) * math.comb(16, 8)


@pytest.mark.parametrize("I,b", [(1, 0), (2, 1), (3, 2), (4, 2), (5, 3), (1000, 10), (1024, 10),
                                 (1025, 11), (5000, 13), (200000, 18), (2 ** 32, 32), (24, 5)])
def test_bits_for_dim(I, b):
    assert oracle.bits_for_dim(I) == b


def test_concatenated_order_is_row_major_index():
    """All bits of mode 0 low, then mode 1, then mode 2: p is the linear index
    i_0 + I'_0 i_1 + I'_0 I'_1 i_2 with I'_n = 2^l(n) (closed form)."""
    dims = [6, 9, 3]
    lbits, _ = oracle.bit_budget(dims)
    order = [0] * lbits[0] + [1] * lbits[1] + [2] * lbits[2]
    rng = np.random.default_rng(0)
    c = np.stack([rng.integers(0, d, 500) for d in dims]).astype(np.uint32)
    lo, hi = oracle.encode(c, dims, order)
    expect = (c[0].astype(np.uint64) + (c[1].astype(np.uint64) << np.uint64(lbits[0]))
              + (c[2].astype(np.uint64) << np.uint64(lbits[0] + lbits[1])))
    assert np.array_equal(lo, expect) and not hi.any()


def _morton3_magic(x):
    """Textbook 3-D Morton code of 10-bit coordinates via magic-number bit spreading."""
    x = x.astype(np.uint64) & np.uint64(0x3FF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x030000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x0300F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x030C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x09249249)
    return x


def test_equal_modes_alto_is_morton():
    """For three 10-bit modes the ALTO order is the Z-order curve with mode 0
    in the lowest bit of each triple."""
    dims = [1000, 1000, 1000]
    order = oracle.alto_order(dims)
    assert list(order) == [0, 1, 2] * 10
    rng = np.random.default_rng(1)
    c = rng.integers(0, 1000, (3, 4000)).astype(np.uint32)
    lo, _ = oracle.encode(c, dims, order)
    expect = _morton3_magic(c[0]) | (_morton3_magic(c[1]) << np.uint64(1)) | (_morton3_magic(c[2]) << np.uint64(2))
    assert np.array_equal(lo, expect)


def test_alto_order_rules():
    dims = [10_000_000, 10_000_000, 1_000_000, 1000, 100]
    lbits, lp = oracle.bit_budget(dims)
    assert lbits == [24, 24, 20, 10, 7] and lp == 85
    order = oracle.alto_order(dims)
    assert oracle.check_order(dims, order)
    # round robin over modes sorted by (l(n), id) with exhausted modes skipped
    assert list(order[:5]) == [4, 3, 2, 0, 1]
    assert list(order[35:40]) == [3, 2, 0, 1, 3]
    assert list(order[47:50]) == [2, 0, 1]
    assert list(order[-4:]) == [0, 1, 0, 1]
    # a mode of length 1 takes no bits
    o = oracle.alto_order([1, 4, 1, 2])
    assert list(o) == [3, 1, 1]


def test_wide_keys_roundtrip_and_bruteforce():
    dims = [2 ** 20, 2 ** 20 + 3, 2 ** 20, 1000, 100]
    lbits, lp = oracle.bit_budget(dims)
    assert lp > 64
    rng = np.random.default_rng(2)
    c = np.stack([rng.integers(0, d, 300) for d in dims]).astype(np.uint32)
    order = list(oracle.alto_order(dims))
    rng.shuffle(order)
    lo, hi = oracle.encode(c, dims, order)
    # pure-Python brute force with big integers
    for e in range(0, 300, 37):
        nxt = [0] * len(dims)
        p = 0
        for t, n in enumerate(order):
            p |= ((int(c[n, e]) >> nxt[n]) & 1) << t
            nxt[n] += 1
        assert p == int(lo[e]) | (int(hi[e]) << 64)
    assert np.array_equal(oracle.decode(lo, hi, dims, order), c)


def test_encode_rejects_bad_inputs():
    dims = [4, 8, 2]
    c = np.array([[0], [0], [2]], dtype=np.uint32)  # i_3 = 2 >= I_3
    with pytest.raises(oracle.OracleError):
        oracle.encode(c, dims, oracle.alto_order(dims))
    c = np.zeros((3, 1), dtype=np.uint32)
    for bad in ([2, 0, 1, 0, 1], [2, 0, 1, 0, 1, 0], [2, 0, 1, 0, 1, 3]):
        assert not oracle.check_order(dims, bad)
        with pytest.raises(oracle.OracleError):
            oracle.encode(c, dims, bad)


def test_sort_is_stable_with_duplicates():
    rng = np.random.default_rng(3)
    dims = [5, 7, 3]
    c = np.stack([rng.integers(0, d, 400) for d in dims]).astype(np.uint32)  # many duplicates
    order = oracle.alto_order(dims)
    lo, hi = oracle.encode(c, dims, order)
    perm = oracle.sort_perm(lo, hi)
    expect = sorted(range(400), key=lambda e: (int(hi[e]), int(lo[e]), e))
    assert perm.tolist() == expect


def _bruteforce_stats(cs, dims, S):
    N, nnz = cs.shape
    P = (nnz + S - 1) // S
    lo = [[min(cs[n, q * S:(q + 1) * S]) for n in range(N)] for q in range(P)]
    hi = [[max(cs[n, q * S:(q + 1) * S]) for n in range(N)] for q in range(P)]
    runs, distinct, maxcount = [], [], []
    for n in range(N):
        r = 0
        for j in range(nnz):
            if j % S == 0 or cs[n, j] != cs[n, j - 1]:
                r += 1
        runs.append(r)
        cnt = {}
        for x in cs[n]:
            cnt[int(x)] = cnt.get(int(x), 0) + 1
        distinct.append(len(cnt))
        maxcount.append(max(cnt.values()))
    return lo, hi, runs, distinct, maxcount


@pytest.mark.parametrize("S", [1, 7, 64, 1000])
def test_partitions_and_stats_bruteforce(S):
    rng = np.random.default_rng(4)
    dims = [50, 300, 6, 2]
    c = np.stack([rng.integers(0, d, 777) for d in dims]).astype(np.uint32)
    enc = oracle.encode_full(c, np.ones(777), dims, S=S)
    lo, hi, runs, distinct, maxcount = _bruteforce_stats(enc["coords"], dims, S)
    assert enc["part_lo"].tolist() == lo and enc["part_hi"].tolist() == hi
    assert enc["runs"].tolist() == runs
    assert enc["distinct"].tolist() == distinct
    assert enc["maxcount"].tolist() == maxcount
    # the sorted stream is non-decreasing in p
    p = [int(a) | (int(b) << 64) for a, b in zip(enc["key_lo"], enc["key_hi"])]
    assert p == sorted(p)
