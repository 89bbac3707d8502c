"""The autotuner's search logic on the CPU (no GPU needed).

The sandbox test follows the paper's sandbox mode (Sec. 4.1.3): rewarded
only for reproducing the ALTO encoding, the search must find it exactly.
"""
import itertools
import math

import pytest

import oracle
from paper_2509_00280_gb300 import tune


@pytest.mark.parametrize("dims", [(4, 8, 2), (1000, 1000, 1000), (200000, 200000, 5000),
                                  (5_000_000, 1_000_000, 100_000, 24), (10 ** 7, 10 ** 7, 10 ** 6, 1000, 100)])
def test_candidates_are_valid_and_alto_matches_the_oracle(dims):
    assert list(tune.alto_order(dims)) == list(oracle.alto_order(dims))
    cands = [tune.alto_order(dims), tune.longest_first(dims)] + [tune.mode_on_top(dims, n) for n in range(len(dims))]
    cands += [tune.block_interleave(dims, b) for b in (2, 4)]
    import random
    rng = random.Random(3)
    cands += [tune.random_interleave(dims, rng) for _ in range(5)]
    for o in cands:
        assert tune.is_valid(o, dims) and oracle.check_order(dims, o)
        for nb in tune.neighbours(o):
            assert oracle.check_order(dims, nb)


def test_mode_on_top_gives_long_runs():
    dims = (4, 8, 2)
    for n in range(3):
        o = tune.mode_on_top(dims, n)
        lb = tune.bit_budget(dims)
        assert list(o[-lb[n]:]) == [n] * lb[n]


@pytest.mark.parametrize("dims", [(4, 8, 2), (16, 64, 8, 4), (200000, 200000, 5000)])
def test_sandbox_recovers_the_alto_order_from_random_starts(dims):
    """Sandbox mode: starting from a random order, with random seeds only
    (the ALTO order is never handed in), the search must reach ALTO exactly."""
    import random
    rng = random.Random(7)
    start = tune.random_interleave(dims, rng)
    seeds = [tune.random_interleave(dims, rng) for _ in range(3)]
    target = tune.alto_order(dims)
    assert start != target and target not in seeds
    res = tune.tune(dims, tune.sandbox_reward(dims), max_evals=20000, patience=20000, baseline_order=start,
                    seeds=seeds)
    assert res.best.order == target
    assert res.best.seconds == 1.0


def test_kendall_distance():
    assert tune.kendall_distance((0, 1, 2), (0, 1, 2)) == 0
    assert tune.kendall_distance((2, 1, 0), (0, 1, 2)) == 3
    assert tune.kendall_distance((1, 0, 0, 1), (0, 0, 1, 1)) == 2


def test_reward_cache_and_patience():
    dims = (4, 8, 2)
    calls = []

    def ev(order, S):
        calls.append((order, S))
        return 1.0, ["x"] * 3  # nothing ever improves

    res = tune.tune(dims, ev, max_evals=100, patience=3)
    assert res.stopped_early and res.evaluations == 4  # baseline + 3 non-improving
    assert len(calls) == len(set(calls)) == res.evaluations
    # every interleaving of the worked example is evaluated at most once
    orders = set(itertools.permutations([0, 0, 1, 1, 1, 2]))
    assert len(orders) == 60

    def ev2(order, S):
        calls.append((order, S))
        return 1.0 + (hash(order) % 97) / 97.0, ["x"] * 3

    calls.clear()
    res = tune.tune(dims, ev2, max_evals=1000, patience=1000)
    assert res.evaluations <= 60 and len(calls) == len(set(calls))
    assert math.isclose(res.best.seconds, min(t.seconds for t in res.trials))


def test_mode_configs_enumerate_the_kernel_plans():
    from paper_2509_00280_gb300 import tune
    dims = (5000, 1000, 100, 24)
    cfgs = tune.mode_configs(dims, 0, 64, "f64")
    # ATOMIC, SEGMENTED flat, then depth 1..2 x 2 level orders x 2 R-tiles, and
    # at depth 2 the Khatri-Rao pair on and off where its table fits: (2, 3) has
    # 2400 rows, (2, 1) 100000 (both fit)
    assert [c.strategy for c in cfgs[:2]] == [1, 2]
    fac = [c for c in cfgs if c.depth > 0]
    assert len(fac) == 2 * 2 * 2 + 2 * 2
    assert {c.level for c in fac} == {(1, 2, 3), (3, 2, 1)}
    assert {c.col_passes for c in fac} == {1, 2}
    assert {(c.depth, c.kr) for c in fac} == {(1, 0), (2, 0), (2, 1)}
    assert not any(c.kr for c in tune.mode_configs(dims, 0, 64, "f32"))
    # the 24-row mode's pair (1, 2) has 1e11 rows, over 2^32
    big = (5_000_000, 1_000_000, 100_000, 24)
    assert not tune.kr_fits(big, (0, 1, 2), 2, 64) and tune.kr_fits(big, (0, 2, 3), 2, 64)
    assert not any(c.kr for c in tune.mode_configs(big, 3, 64, "f64") if c.level == (0, 1, 2))
    # a 24-row output fits shared memory: PRIVATIZED is tried
    assert any(c.strategy == 3 for c in tune.mode_configs(dims, 3, 64, "f32"))
    # 3-mode tensors: one level; R = 12 in FP32 cannot be halved into whole 4-element vectors
    cfgs3 = tune.mode_configs((300, 200, 100), 1, 12, "f32")
    assert {c.depth for c in cfgs3 if c.strategy == 2} == {0, 1}
    assert all(c.col_passes == 1 for c in cfgs3)
    # 2-mode and 6-mode tensors have no factored plans
    assert all(c.depth == 0 for c in tune.mode_configs((300, 200), 0, 16, "f32"))
