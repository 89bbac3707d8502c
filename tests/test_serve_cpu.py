"""Host logic of the CP-ALS service: admission by device footprint, the
bounded bypass of a waiting head, percentiles, the request recipe, and the
library's host-only footprint query. No GPU."""
import math
import random
import threading
import time

import numpy as np
import pytest

import synth
from paper_2509_00280_gb300.serve import AdmissionQueue, percentile


def test_fifo_when_everything_fits():
    q = AdmissionQueue(100)
    for k in range(5):
        q.put(k, 10)
    got = [q.take(timeout=1)[0] for _ in range(5)]
    assert got == [0, 1, 2, 3, 4]
    assert q.in_use == 50 and q.peak_in_use == 50


def test_oversized_request_is_refused():
    q = AdmissionQueue(100)
    with pytest.raises(ValueError):
        q.put("big", 101)
    q.put("ok", 100)
    assert q.take(timeout=1) == ("ok", 100)


def test_head_that_does_not_fit_is_bypassed_a_bounded_number_of_times():
    q = AdmissionQueue(100, max_bypass=2)
    q.put("a", 60)
    assert q.take(timeout=1)[0] == "a"          # 60 in use
    q.put("head", 50)                           # does not fit (40 free)
    for k in range(4):
        q.put(f"s{k}", 10)
    assert q.take(timeout=1)[0] == "s0"         # bypass 1
    assert q.take(timeout=1)[0] == "s1"         # bypass 2
    assert q.take(timeout=0.05) is None         # no third bypass: head waits
    q.release(60)                                # "a" done: 80 free
    assert q.take(timeout=1)[0] == "head"
    assert q.take(timeout=1)[0] == "s2"


def test_close_wakes_takers_and_drains():
    q = AdmissionQueue(10)
    q.put("x", 5)
    q.close()
    assert q.take(timeout=1)[0] == "x"
    assert q.take(timeout=1) is None
    with pytest.raises(RuntimeError):
        q.put("y", 1)


def test_budget_never_exceeded_under_concurrent_workers():
    rng = random.Random(5)
    budget = 1000
    q = AdmissionQueue(budget, max_bypass=3)
    sizes = [rng.randint(1, budget) for _ in range(200)]
    seen, lock, over = [], threading.Lock(), []

    def worker():
        while True:
            got = q.take()
            if got is None:
                return
            item, nbytes = got
            with lock:
                if q.in_use > budget:
                    over.append(q.in_use)
                seen.append(item)
            time.sleep(rng.random() * 1e-3)
            q.release(nbytes)

    ts = [threading.Thread(target=worker) for _ in range(6)]
    for t in ts:
        t.start()
    for k, s in enumerate(sizes):
        q.put(k, s)
    q.close()
    for t in ts:
        t.join(timeout=60)
    assert sorted(seen) == list(range(200))
    assert not over and q.peak_in_use <= budget and q.in_use == 0


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    assert percentile([7.0], 99) == 7.0
    assert math.isnan(percentile([], 50))
    assert percentile([3, 1, 2], 50) == 2


def test_request_recipe_ranges_and_determinism():
    Ns, Rs = set(), set()
    for i in range(300):
        spec, R = synth.serving_request(i)
        assert spec == synth.serving_request(i)[0]
        N = len(spec.dims)
        Ns.add(N)
        Rs.add(R)
        assert 1e4 - 1 <= spec.nnz <= 2e7 + 1
        assert all(100 <= d <= 1_000_000 for d in spec.dims)
        alpha = spec.dists[0][1]
        assert 1.0 <= alpha <= 1.4 and all(d == ("zipf", alpha) for d in spec.dists)
    assert Ns == {3, 4, 5} and Rs == {8, 16, 32, 64}
    # nnz log-uniform: the median of log10(nnz) is near the middle of [4, 7.3]
    med = np.median([math.log10(synth.serving_request(i)[0].nnz) for i in range(300)])
    assert abs(med - 0.5 * (4 + math.log10(2e7))) < 0.35


def test_distinct_once_keeps_first_draws():
    spec, _ = synth.serving_request(5, nnz_range=(3e4, 3e4 + 1))
    c, v = synth.make_tensor(spec)
    tuples = set(map(tuple, c.T.tolist()))
    assert len(tuples) == c.shape[1] <= spec.nnz      # distinct
    allc = synth._draw_coords(spec, 0, spec.nnz, [synth.zipf_table(int(I), d[1]) for I, d in
                                                    zip(spec.dims, spec.dists)])
    allv = synth.make_values(spec)
    firsts, seen = [], set()
    for e in range(spec.nnz):
        t = tuple(allc[:, e].tolist())
        if t not in seen:
            seen.add(t)
            firsts.append(e)
    assert np.array_equal(c, allc[:, firsts]) and np.array_equal(v, allv[firsts])


def test_poisson_arrivals_rate():
    a = synth.poisson_arrivals(20000, 50.0, seed=0)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 20000 - 1 / 50.0) < 0.03 / 50.0 * 10


def test_footprint_is_host_only_and_consistent():
    from paper_2509_00280_gb300 import build_lib
    build_lib.build()
    import paper_2509_00280_gb300 as rl
    small = rl.relate_footprint((1000, 1000, 1000), 1_000_000, 16)
    big = rl.relate_footprint((1000, 1000, 1000), 2_000_000, 16)
    assert small["encode_peak"] > small["resident"] > 0
    assert big["resident"] > small["resident"] and big["encode_peak"] > small["encode_peak"]
    # 30 key bits -> 4-byte words; 5 x 20 bits -> 16-byte words
    w4 = rl.relate_footprint((1000, 1000, 1000), 1_000_000, 16)["resident"]
    w16 = rl.relate_footprint((2 ** 20,) * 5, 1_000_000, 16)["resident"]
    assert w16 - w4 > 12 * 1_000_000
    f32 = rl.relate_footprint((1000, 2000, 3000), 10_000, 8, factor_dtype="f32")
    f64 = rl.relate_footprint((1000, 2000, 3000), 10_000, 8, factor_dtype="f64")
    assert f32["factors"] == 6000 * 8 * 4 and f64["factors"] == 2 * f32["factors"]
    assert rl.relate_footprint((1000, 2000, 3000), 10_000, 64)["cpals_workspace"] > f32["cpals_workspace"]
    dev = rl.relate_footprint((1000, 1000, 1000), 1_000_000, 16, coords_on_device=True)
    assert small["encode_peak"] - dev["encode_peak"] == 1_000_000 * (3 * 4 + 4)
    # FP64 factors, 4 modes: the AUTO plans' Khatri-Rao table (the two shortest
    # other modes of a mode, I_a * I_b <= nnz / 4 rows) joins the workspace:
    # 60000 rows (modes 1 and 3 for mode 2) at 400K nonzeros, 6000 (modes 2 and 3) at 100K
    d4 = (6000, 3000, 300, 20)
    ws = {(dt, z): rl.relate_footprint(d4, z, 16, factor_dtype=dt)["cpals_workspace"]
          for dt in ("f64", "f32") for z in (100_000, 400_000)}
    assert ws["f64", 400_000] - ws["f64", 100_000] == (60000 - 6000) * 16 * 8
    assert ws["f32", 400_000] == ws["f32", 100_000]
    with pytest.raises(rl.RelateError):
        rl.relate_footprint((2 ** 33, 4), 10, 8)
    with pytest.raises(rl.RelateError):
        rl.relate_footprint((10, 10), 10, 65)


def test_with_precision_keeps_the_tensor_and_widens_fp64_values():
    import numpy as np
    from paper_2509_00280_gb300.serve import Request, with_precision
    c = np.zeros((3, 5), dtype=np.uint32)
    v = np.arange(5, dtype=np.float32)
    reqs = [Request(c, v, (4, 4, 4), 8, rid=0)]
    f64 = with_precision(reqs, "f64")[0]
    assert f64.precision == "f64" and f64.vals.dtype == np.float64 and np.array_equal(f64.vals, v)
    assert f64.coords is c and reqs[0].precision == "f32" and reqs[0].vals.dtype == np.float32
    bf = with_precision(reqs, "bf16")[0]
    assert bf.precision == "bf16" and bf.vals is v
