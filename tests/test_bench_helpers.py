"""Host-side arithmetic of bench.py (no GPU): the roofline's algorithmic bytes
(the compulsory traffic of one mode-n MTTKRP: the stream once, each distinct
row of the other factors once, the output once), the per-step launch count
(checked against an ncu launch list of the 150M-nonzero FP64 workload: 499
kernels per step, 143 of them the encode) and the scaling of the cache
traffic table."""
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


STATS = {"nmodes": 3, "lp": 49, "nnz": 50_000_000, "key_bytes": 8,
         "distinct": [170_000, 160_000, 5000], "dims": [200_000, 200_000, 5000]}


def test_algorithmic_bytes_by_hand():
    R, fb, ab, vb = 32, 4, 4, 4
    got = bench._algorithmic_bytes(STATS, 0, R, fb, ab, vb)
    want = 50_000_000 * (8 + 4) + (160_000 + 5000) * 32 * 4 + 200_000 * 32 * 4
    assert got == want
    # FP64: 8-byte factor rows, output and values
    assert bench._algorithmic_bytes(STATS, 2, R, 8, 8, 8) == \
        50_000_000 * 16 + (170_000 + 160_000) * 32 * 8 + 5000 * 32 * 8


def test_launch_count_matches_the_launch_list():
    # encode: key build, 5 kernels x (7 key passes + 3 x 4 count passes), words,
    # gather, statistics, 3 x (summary, count, hot rows), norm (2) = 110
    # CP-ALS FP32: 3 x 2 initial Gram kernels + 3 tile orders + 25 x (7 x 3 + fit + record)
    assert bench._launches_per_step(STATS, 25, "f32", 3, 32) == 110 + 6 + 3 + 25 * 23
    bf16 = bench._launches_per_step(STATS, 10, "bf16", 3, 16)
    assert bf16 == 110 + 6 + 3 + 10 * (9 * 3 + 2)
    # the 150M-nonzero 4-mode FP64 workload (l(p) = 65: 9 key passes), counted
    # in its ncu launch list: encode 143; CP-ALS 4 x 3 initial Gram kernels,
    # 4 tile orders, 10 x (8 x 4 + 2)
    s4 = {"nmodes": 4, "lp": 65}
    assert bench._launches_per_step(s4, 10, "f64", 4, 64) == 143 + 12 + 4 + 340 == 499
    # its dims: only the 24-row mode is small enough for the FP64 pipe
    s4d = dict(s4, dims=[5_000_000, 1_000_000, 100_000, 24])
    assert bench._launches_per_step(s4d, 10, "f64", 4, 64) == 499 - 1 - 10
    # modes 0 and 1 fuse the pair (2, 3): one table per iteration, reused by mode 1
    assert bench._launches_per_step(s4d, 10, "f64", 4, 64, [[2, 3], [2, 3], None, None]) == 499 - 1
    assert bench._kr_builds([[2, 3], [2, 3], [1, 3], None]) == 2
    assert bench._kr_builds([[1, 2], None, None, [1, 2]]) == 2  # mode 1 rewrote A_1 in between
    assert bench._kr_builds([[1, 2], [0, 2], None]) == 2        # another pair


def test_cache_rates_scale_with_nonzeros(monkeypatch):
    sha = bench._kernel_sha()
    monkeypatch.setattr(bench, "NCU_CACHE", [{"sha256": sha, "family": "fam-x", "dtype": "f64", "workload": "fam-x-1M",
                                              "nnz": 1e6, "l1_bytes": 2e9, "l2_bytes": 1e9}])
    r = bench._cache_rates("f64", "fam-x-5M", 5e6, 0.5)
    assert abs(r["l1_gbs"] - 2e9 * 5 / 0.5 / 1e9) < 1e-9 and abs(r["l2_gbs"] - 1e9 * 5 / 0.5 / 1e9) < 1e-9
    assert bench._cache_rates("f32", "fam-x-5M", 5e6, 0.5) is None      # other precision
    assert bench._cache_rates("f64", "other-5M", 5e6, 0.5) is None      # other family
    monkeypatch.setattr(bench, "NCU_CACHE", [dict(bench.NCU_CACHE[0], sha256="0" * 64)])
    assert bench._cache_rates("f64", "fam-x-5M", 5e6, 0.5) is None      # counters of another kernel


def test_kernel_sha_ignores_comments(tmp_path, monkeypatch):
    import shutil
    src = tmp_path / "paper_2509_00280_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in ("mttkrp_impl.cuh", "mttkrp.cu", "mttkrp_fac.cuh"):
        shutil.copy(f"{ROOT}/paper_2509_00280_gb300/csrc/{name}", src / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench._kernel_sha()
    p = src / "mttkrp.cu"
    p.write_text(p.read_text() + "\n// a comment\n/* another\n one */\n\n")
    assert bench._kernel_sha() == a
    p.write_text(p.read_text() + "\nint x_unused_for_the_test;\n")
    assert bench._kernel_sha() != a
