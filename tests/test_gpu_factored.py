"""The fiber-factored SEGMENTED MTTKRP (relate_set_mode_plan) against the CPU
oracle (Sec. 2.2, Fig. 2: the same per-nonzero terms, regrouped by
distributivity over fibers of equal (i_n, i_p1..i_pl) inside sorted tiles).

Tolerances as every MTTKRP test (relative Frobenius error against the FP64
oracle on the same inputs): FP64 <= 1e-12, FP32 <= 1e-5, BF16 factors <= 1e-5
against the oracle fed the BF16-rounded factors; integer-exact inputs bit for
bit. Covered: 3, 4 and 5 modes, every depth 0..N-2, AUTO and explicit level
orders, one and two column passes, skewed modes whose hottest rows go to the
per-block copies, ragged and tiny partitions.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, TORCH_DT, encode_dev, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5}
SEG = rl.RELATE_CONFLICT_SEGMENTED


def _factors(dims, R, fdt, seed=5, kind="uniform"):
    fs = synth.init_factors(dims, R, seed=seed, kind=kind)
    if fdt == "bf16":
        fs = [oracle.round_bf16(f.astype(np.float32)).astype(np.float64) for f in fs]
    elif fdt == "f32":
        fs = [f.astype(np.float32).astype(np.float64) for f in fs]
    dfs = [torch.from_numpy(f).to(DEV).to(TORCH_DT[fdt]).contiguous() for f in fs]
    return fs, dfs


def _run(h, n, dfs, R, fdt):
    out = torch.empty((h.dims[n], R), dtype=torch.float64 if fdt == "f64" else torch.float32, device=DEV)
    rl.relate_mttkrp(h, n, dfs, R, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def t4():
    spec = synth.TensorSpec("fac4d", (20000, 5000, 700, 24), 400_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="uniform", value_dtype="f32", seed=51)
    c, v = synth.make_tensor(spec)
    return spec, c, v


@pytest.mark.parametrize("fdt", ["f64", "f32", "bf16"])
def test_four_modes_every_depth_order_and_pass(t4, fdt):
    spec, c, v = t4
    R = 32
    h = encode_dev(c, v.astype(np.float64) if fdt == "f64" else v, spec.dims, factor_dtype=fdt)
    fs, dfs = _factors(spec.dims, R, fdt)
    refs = [oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs) for n in range(4)]
    for n in range(4):
        rl.relate_set_conflict(h, n, SEG)
        # AUTO: N - 2 levels for FP64 (bound by the FP64 pipe), the flat loop for FP32 / BF16
        assert rl.relate_get_mode_plan(h, n, R)["depth"] == (2 if fdt == "f64" else 0)
        others = [k for k in range(4) if k != n]
        for depth, level, passes in ((0, None, 1), (1, None, 1), (2, None, 1), (2, others[::-1], 1),
                                     (1, [others[1], others[2], others[0]], 2), (2, None, 2)):
            rl.relate_set_mode_plan(h, n, depth, level, passes)
            plan = rl.relate_get_mode_plan(h, n, R)
            assert plan["depth"] == depth and plan["col_passes"] == passes
            if level is not None:
                assert plan["level"] == list(level)
            got = _run(h, n, dfs, R, fdt)
            assert rel_fro(got, refs[n]) <= TOL[fdt], (fdt, n, depth, level, passes)
    rl.relate_sync_status(h)
    h.close()


@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_three_modes_skewed_with_hot_row_copies(fdt):
    # Zipf 1.2 on 2M nonzeros: the hottest rows hold >= 2^15 nonzeros, so the
    # per-block copies of the hot rows are in use
    spec = synth.scaled(synth.WORKLOADS["zipf3d-200Kx200Kx5K-50M"]["spec"], 2_000_000)
    c, v = synth.make_tensor(spec)
    R = 32
    h = encode_dev(c, v.astype(np.float64) if fdt == "f64" else v, spec.dims, factor_dtype=fdt)
    st = rl.relate_get_stats(h)
    assert max(st["maxcount"]) >= 2 ** 15
    fs, dfs = _factors(spec.dims, R, fdt)
    for n in range(3):
        rl.relate_set_conflict(h, n, SEG)
        rl.relate_set_mode_plan(h, n, 1)
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
        assert rel_fro(_run(h, n, dfs, R, fdt), ref) <= TOL[fdt], (fdt, n)
    h.close()


@pytest.mark.parametrize("fdt", ["f64", "bf16"])
def test_five_modes_every_depth(fdt):
    spec = synth.TensorSpec("fac5d", (3000, 3000, 400, 100, 30), 300_000, (("zipf", 1.3),) * 2 + (("uniform",),) * 3,
                            values="uniform", value_dtype="f32", seed=52)
    c, v = synth.make_tensor(spec)
    R = 16
    h = encode_dev(c, v.astype(np.float64) if fdt == "f64" else v, spec.dims, factor_dtype=fdt)
    fs, dfs = _factors(spec.dims, R, fdt)
    for n in (0, 3):
        rl.relate_set_conflict(h, n, SEG)
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
        for depth in (1, 2, 3):
            rl.relate_set_mode_plan(h, n, depth)
            assert rel_fro(_run(h, n, dfs, R, fdt), ref) <= TOL[fdt], (fdt, n, depth)
    h.close()


@pytest.mark.parametrize("S", [4100, 12, 2048])
def test_ragged_and_tiny_partitions(S):
    spec = synth.TensorSpec("fac4d-ragged", (900, 700, 60, 24), 100_003, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="uniform", value_dtype="f64", seed=53)
    c, v = synth.make_tensor(spec)
    R = 16
    h = encode_dev(c, v, spec.dims, factor_dtype="f64", partition_size=S)
    fs, dfs = _factors(spec.dims, R, "f64")
    for n in range(4):
        rl.relate_set_conflict(h, n, SEG)
        rl.relate_set_mode_plan(h, n, 2, None, 2)
        ref = oracle.mttkrp(c, v, spec.dims, n, fs)
        assert rel_fro(_run(h, n, dfs, R, "f64"), ref) <= 1e-12, (S, n)
    h.close()


def test_integer_exact_factored_sums_bitwise():
    """Integer values and factors keep every partial sum exact in FP64, so the
    regrouped sums equal the oracle's bit for bit."""
    spec = synth.TensorSpec("fac-int4d", (80, 60, 40, 9), 150_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="int:1:8", value_dtype="f64", seed=54)
    c, v = synth.make_tensor(spec)
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=3, kind="int:0:4")
    dfs = [torch.from_numpy(f).to(DEV).contiguous() for f in fs]
    h = encode_dev(c, v, spec.dims, factor_dtype="f64")
    for n in range(4):
        rl.relate_set_conflict(h, n, SEG)
        for depth in (1, 2):
            rl.relate_set_mode_plan(h, n, depth)
            assert np.array_equal(_run(h, n, dfs, R, "f64"), oracle.mttkrp(c, v, spec.dims, n, fs)), (n, depth)
    h.close()


def test_plan_validation():
    spec = synth.TensorSpec("plan3d", (50, 40, 30), 5000, (("uniform",),) * 3, seed=55)
    c, v = synth.make_tensor(spec)
    h = encode_dev(c, v, spec.dims)
    for bad in (dict(depth=-2), dict(level=[0, 1]), dict(level=[1, 1]), dict(col_passes=-1)):
        with pytest.raises(rl.RelateError):
            rl.relate_set_mode_plan(h, 0, **bad)
    rl.relate_set_mode_plan(h, 0, 1, [2, 1], 1)
    assert rl.relate_get_mode_plan(h, 0, 8)["level"] == [2, 1]
    h.close()


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_khatri_rao_pair_on_off(t4, n):
    """The fused Khatri-Rao pair (relate_set_mode_kr): the deepest level's
    mode and the innermost one as one slot over the rows of their Khatri-Rao
    product (Sec. 2.2), against the oracle and against the unfused kernel."""
    spec, c, v = t4
    R = 32
    h = encode_dev(c, v.astype(np.float64), spec.dims, factor_dtype="f64")
    fs, dfs = _factors(spec.dims, R, "f64")
    ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
    rl.relate_set_conflict(h, n, SEG)
    others = sorted((k for k in range(4) if k != n), key=lambda k: -spec.dims[k])
    rows = spec.dims[others[1]] * spec.dims[others[2]]
    got = rl.relate_get_mode_kr(h, n, R)
    assert got == ({"kr": 1, "rows": rows} if rows * 4 <= spec.nnz else {"kr": 0, "rows": 0})
    res = {}
    for kr in (0, 1):
        rl.relate_set_mode_kr(h, n, kr)
        assert rl.relate_get_mode_kr(h, n, R)["kr"] == kr
        res[kr] = _run(h, n, dfs, R, "f64")
        assert rel_fro(res[kr], ref) <= 1e-12, (n, kr)
    assert rel_fro(res[1], res[0]) <= 1e-13
    # depth 1 leaves two unfactored slots: no pair to fuse
    rl.relate_set_mode_plan(h, n, 1)
    assert rl.relate_get_mode_kr(h, n, R)["kr"] == 0
    assert rel_fro(_run(h, n, dfs, R, "f64"), ref) <= 1e-12
    with pytest.raises(rl.RelateError):
        rl.relate_set_mode_kr(h, n, 2)
    h.close()


def test_khatri_rao_pair_five_modes_and_factor_updates():
    """Five modes at depth 3 (the kernel then runs 4 slots at depth 2); the
    table is rebuilt on every relate_mttkrp call, so changed factors are seen."""
    spec = synth.TensorSpec("kr5d", (3000, 2500, 400, 60, 30), 300_000,
                            (("zipf", 1.2),) * 2 + (("uniform",),) * 3, values="uniform", value_dtype="f32", seed=57)
    c, v = synth.make_tensor(spec)
    R = 16
    h = encode_dev(c, v.astype(np.float64), spec.dims, factor_dtype="f64")
    fs, dfs = _factors(spec.dims, R, "f64")
    for n in (0, 4):
        rl.relate_set_conflict(h, n, SEG)
        rl.relate_set_mode_kr(h, n, 1)
        assert rl.relate_get_mode_kr(h, n, R)["kr"] == 1
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fs)
        assert rel_fro(_run(h, n, dfs, R, "f64"), ref) <= 1e-12, n
    # scale the innermost factor of mode 0's pair: the next call rebuilds the table
    k = int(np.argmin([spec.dims[i] for i in range(1, 5)])) + 1
    fs[k] = fs[k] * 3.0
    dfs[k].mul_(3.0)
    ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, 0, fs)
    assert rel_fro(_run(h, 0, dfs, R, "f64"), ref) <= 1e-12
    h.close()
