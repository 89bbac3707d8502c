"""GPU MTTKRP vs the CPU oracle (Sec. 2.2, Fig. 2).

Tolerances (relative Frobenius error against the FP64 oracle on the same
inputs): FP64 <= 1e-12; FP32 <= 1e-5; BF16 factors <= 1e-5 against the
oracle fed the BF16-rounded factors (the arithmetic itself is FP32) and
<= 2e-2 against the unrounded factors. Integer-exact inputs must match
bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, encode_dev, factors_dev, mttkrp_dev, rel_fro

pytestmark = pytest.mark.gpu

STRATS = {"atomic": rl.RELATE_CONFLICT_ATOMIC, "segmented": rl.RELATE_CONFLICT_SEGMENTED,
          "privatized": rl.RELATE_CONFLICT_PRIVATIZED}


def _tensor(name, nnz=None, dims=None, value_dtype=None):
    spec = synth.WORKLOADS[name]["spec"]
    if nnz is not None or dims is not None:
        spec = synth.scaled(spec, nnz or spec.nnz, dims=dims)
    if value_dtype:
        spec.value_dtype = value_dtype
    c, v = synth.make_tensor(spec)
    return spec, c, v


@pytest.fixture(scope="module")
def cfg_uniform():
    spec, c, v = _tensor("uniform3d-1000x1000x1000-1M")
    fs = synth.init_factors(spec.dims, 16, seed=0)
    refs = [oracle.mttkrp(c, v, spec.dims, n, fs) for n in range(3)]
    return spec, c, v, fs, refs


@pytest.mark.parametrize("strategy", ["auto", "atomic", "segmented", "privatized"])
def test_fp64_uniform_1M_all_modes(cfg_uniform, strategy):
    spec, c, v, fs, refs = cfg_uniform
    h = encode_dev(c, v, spec.dims, factor_dtype="f64")
    if strategy != "auto":
        for n in range(3):
            rl.relate_set_conflict(h, n, STRATS[strategy])
    dfs = factors_dev(fs, "f64")
    for n in range(3):
        got = mttkrp_dev(h, n, dfs, 16, acc="f64")
        assert rel_fro(got, refs[n]) <= 1e-12, (n, strategy)
    rl.relate_sync_status(h)  # no bounded wait gave up
    h.close()


def test_integer_exact_bitwise():
    spec = synth.TensorSpec("int4d", (60, 50, 40, 7), 200_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="int:1:8", value_dtype="f64", seed=11)
    c, v = synth.make_tensor(spec)
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=3, kind="int:0:4")
    for fdt, acc in (("f64", "f64"), ("f32", "f32")):
        h = encode_dev(c, v if fdt == "f64" else v.astype(np.float32), spec.dims, factor_dtype=fdt)
        for strat in ("atomic", "segmented", "privatized"):
            for n in range(4):
                rl.relate_set_conflict(h, n, STRATS[strat])
            dfs = factors_dev(fs, fdt)
            for n in range(4):
                ref = oracle.mttkrp(c, v, spec.dims, n, fs)
                if fdt == "f32" and np.abs(ref).max() >= 2 ** 24:
                    continue
                got = mttkrp_dev(h, n, dfs, R, acc=acc)
                assert np.array_equal(got, ref), (fdt, strat, n)
        h.close()


@pytest.mark.parametrize("fdt", ["f32", "bf16"])
def test_zipf3d_fp32_bf16(fdt):
    spec, c, v = _tensor("zipf3d-200Kx200Kx5K-50M", nnz=2_000_000)
    R = 32
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float32)
    v64 = v.astype(np.float64)
    h = encode_dev(c, v, spec.dims, factor_dtype=fdt)
    dfs = factors_dev(fs, fdt)
    for n in range(3):
        got = mttkrp_dev(h, n, dfs, R)
        if fdt == "f32":
            ref = oracle.mttkrp(c, v64, spec.dims, n, [f.astype(np.float64) for f in fs])
            assert rel_fro(got, ref) <= 1e-5, n
        else:
            fr = [oracle.round_bf16(f).astype(np.float64) for f in fs]
            ref_r = oracle.mttkrp(c, v64, spec.dims, n, fr)
            ref_u = oracle.mttkrp(c, v64, spec.dims, n, [f.astype(np.float64) for f in fs])
            assert rel_fro(got, ref_r) <= 1e-5, n
            assert rel_fro(got, ref_u) <= 2e-2, n
    h.close()


@pytest.mark.parametrize("name,nnz,R,fdt", [
    ("zipf4d-5Mx1Mx100Kx24-150M", 300_000, 64, "f32"),
    ("zipf5d-10Mx10Mx1Mx1Kx100-100M", 300_000, 16, "bf16"),
    ("zipf5d-10Mx10Mx1Mx1Kx100-100M", 100_000, 16, "f64"),
])
def test_wide_keys_4d_5d(name, nnz, R, fdt):
    spec, c, v = _tensor(name, nnz=nnz)
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float32)
    v64 = v.astype(np.float64)
    vin = v64 if fdt == "f64" else v
    h = encode_dev(c, vin, spec.dims, factor_dtype=fdt)
    dfs = factors_dev(fs, fdt)
    N = len(spec.dims)
    fr = [oracle.round_bf16(f).astype(np.float64) for f in fs] if fdt == "bf16" else [f.astype(np.float64) for f in fs]
    tol = 1e-12 if fdt == "f64" else 1e-5
    for n in range(N):
        got = mttkrp_dev(h, n, dfs, R, acc="f64" if fdt == "f64" else "f32")
        ref = oracle.mttkrp(c, v64, spec.dims, n, fr)
        assert rel_fro(got, ref) <= tol, (n, rl.relate_get_conflict(h, n, R))
    h.close()


@pytest.mark.parametrize("R", [1, 5, 13, 33, 64])
@pytest.mark.parametrize("fdt", ["f64", "f32", "bf16"])
def test_odd_ranks_scalar_and_vector_paths(R, fdt):
    rng = np.random.default_rng(R)
    dims = (300, 77, 1200)
    c = np.stack([rng.integers(0, d, 40000) for d in dims]).astype(np.uint32)
    v = rng.random(40000)
    fs = [rng.random((d, R)) for d in dims]
    h = encode_dev(c, v if fdt == "f64" else v.astype(np.float32), dims, factor_dtype=fdt)
    dfs = factors_dev(fs, fdt)
    fr = fs if fdt != "bf16" else [oracle.round_bf16(f.astype(np.float32)).astype(np.float64) for f in fs]
    vr = v if fdt == "f64" else v.astype(np.float32).astype(np.float64)
    fr = fr if fdt != "f32" else [f.astype(np.float32).astype(np.float64) for f in fs]
    tol = 1e-12 if fdt == "f64" else 1e-5
    for strat in ("atomic", "segmented", "privatized"):
        for n in range(3):
            rl.relate_set_conflict(h, n, STRATS[strat])
        for n in range(3):
            got = mttkrp_dev(h, n, dfs, R, acc="f64" if fdt == "f64" else "f32")
            ref = oracle.mttkrp(c, vr, dims, n, fr)
            assert rel_fro(got, ref) <= tol, (strat, n)
    h.close()


def test_two_modes_and_bit_order_invariance():
    rng = np.random.default_rng(9)
    dims = (5000, 3000)
    c = np.stack([rng.integers(0, d, 100000) for d in dims]).astype(np.uint32)
    v = rng.random(100000)
    R = 16
    fs = [rng.random((d, R)) for d in dims]
    refs = [oracle.mttkrp(c, v, dims, n, fs) for n in range(2)]
    order = list(oracle.alto_order(dims))
    for trial in range(3):
        h = encode_dev(c, v, dims, factor_dtype="f64", bit_order=np.array(order, dtype=np.int8))
        dfs = factors_dev(fs, "f64")
        for n in range(2):
            assert rel_fro(mttkrp_dev(h, n, dfs, R, acc="f64"), refs[n]) <= 1e-12
        h.close()
        rng.shuffle(order)


def test_gram():
    rng = np.random.default_rng(12)
    for I, R in ((1, 1), (1000, 16), (77777, 64), (200000, 32)):
        A = rng.random((I, R))
        G = torch.empty((R, R), dtype=torch.float64, device=DEV)
        for dt in ("f64", "f32", "bf16"):
            t = factors_dev([A], dt)[0]
            rl.relate_gram(t, R, dt, G)
            torch.cuda.synchronize()
            Ar = t.to(torch.float64).cpu().numpy()
            ref = oracle.gram(Ar)
            # FP32/BF16 inputs accumulate in FP32 over a block's rows (I/304 of
            # them, <= 660 here): worst case ~660 * 2^-24 = 4e-5, typical
            # sqrt(660) * 2^-24 = 1.5e-6 relative; FP64 inputs stay in FP64
            tol = 1e-13 if dt == "f64" else 2e-5
            assert rel_fro(G.cpu().numpy(), ref) <= tol, (I, R, dt)


@pytest.mark.parametrize("I,R", [(1, 8), (127, 24), (128, 40), (129, 56), (5000, 64), (100_003, 32), (0, 16)])
def test_gram_bf16_tensor_cores_exact_on_integers(I, R):
    """BF16 inputs (R a multiple of 8) run on the tcgen05 tensor cores. With
    small integer entries every product and partial sum is exact in FP32, so
    the result must equal the exact integer Gram bit for bit."""
    rng = np.random.default_rng(I + R)
    A = rng.integers(-3, 4, (I, R)).astype(np.float64)
    t = factors_dev([A], "bf16")[0] if I else torch.zeros((0, R), dtype=torch.bfloat16, device=DEV)
    G = torch.full((R, R), float("nan"), dtype=torch.float64, device=DEV)
    rl.relate_gram(t, R, "bf16", G)
    torch.cuda.synchronize()
    assert np.array_equal(G.cpu().numpy(), A.T @ A)


@pytest.fixture(scope="module")
def skewed():
    """A tensor whose mode 0 has a row with ~40% of the nonzeros (so the
    SEGMENTED kernel keeps per-block copies of its hot rows), and oracle
    results per factor precision."""
    spec = synth.TensorSpec("skewed3d", (50_000, 3000, 800), 400_000,
                            (("zipf", 1.6), ("zipf", 1.1), ("zipf", 1.1)), seed=31)
    c, v = synth.make_tensor(spec)
    R = 32
    fs = synth.init_factors(spec.dims, R, seed=3, dtype=np.float32)
    refs = {}
    for fdt in ("f64", "f32", "bf16"):
        fr = [oracle.round_bf16(f).astype(np.float64) for f in fs] if fdt == "bf16" else \
             [f.astype(np.float64) for f in fs]
        refs[fdt] = [oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, fr) for n in range(3)]
    return spec, c, v, fs, R, refs


@pytest.mark.parametrize("S", [2048, 3000, 1001, 8192])
@pytest.mark.parametrize("fdt", ["f64", "f32", "bf16"])
def test_segmented_tile_order_partition_sizes(skewed, S, fdt):
    """The SEGMENTED kernel with its precomputed tile order and hot-row copies,
    at partition sizes that give ragged tiles (3000, 8192), one tile per
    partition (2048) and partitions that are not a multiple of 4 nonzeros
    (1001: plain loads instead of TMA copies)."""
    spec, c, v, fs, R, refs = skewed
    vin = v.astype(np.float64) if fdt == "f64" else v
    h = encode_dev(c, vin, spec.dims, factor_dtype=fdt, partition_size=S)
    st = rl.relate_get_stats(h)
    assert st["maxcount"][0] >= 1 << 15  # mode 0 takes the hot-row copies
    for n in range(3):
        rl.relate_set_conflict(h, n, rl.RELATE_CONFLICT_SEGMENTED)
    dfs = factors_dev(fs, fdt)
    tol = 1e-12 if fdt == "f64" else 1e-5
    for n in range(3):
        got = mttkrp_dev(h, n, dfs, R, acc="f64" if fdt == "f64" else "f32")
        assert rel_fro(got, refs[fdt][n]) <= tol, (S, fdt, n)
        again = mttkrp_dev(h, n, dfs, R, acc="f64" if fdt == "f64" else "f32")  # tile order reused
        assert rel_fro(again, refs[fdt][n]) <= tol, (S, fdt, n)
    h.close()


@pytest.mark.parametrize("dims", [(20, 30, 40, 50, 60, 70), (5, 6, 7, 8, 9, 10, 11, 12)])
def test_six_and_eight_modes(dims):
    """N > 5 runs the generic instantiation (runtime N) of every strategy."""
    rng = np.random.default_rng(len(dims))
    nnz = 30_000
    c = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    v = rng.random(nnz)
    R = 16
    fs = [rng.random((d, R)) for d in dims]
    refs = [oracle.mttkrp(c, v, dims, n, fs) for n in range(len(dims))]
    h = encode_dev(c, v, dims, factor_dtype="f64")
    dfs = factors_dev(fs, "f64")
    for strat in ("auto", "atomic", "segmented", "privatized"):
        for n in range(len(dims)):
            if strat != "auto":
                rl.relate_set_conflict(h, n, STRATS[strat])
            assert rel_fro(mttkrp_dev(h, n, dfs, R, acc="f64"), refs[n]) <= 1e-12, (strat, n)
    h.close()
