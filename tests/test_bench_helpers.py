"""Host-side arithmetic of bench.py (no GPU): the roofline's algorithmic bytes
(the compulsory traffic of one mode-n MTTKRP: the stream once, each distinct
row of the other factors once, the output once) and the per-step launch count
(checked against an ncu launch list of the 50M-nonzero workload: 594 kernels
per step without graph replay of fixed-count iterations, 619 with it)."""
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
    # CP-ALS: 3 x 2 initial Gram kernels + 3 tile orders + 25 x (6 x 3 + fit + record)
    assert bench._launches_per_step(STATS, 25, "f32", 3, 32) == 110 + 6 + 3 + 25 * 20
    bf16 = bench._launches_per_step(STATS, 10, "bf16", 3, 16)
    assert bf16 == 110 + 6 + 3 + 10 * (9 * 3 + 2)


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
