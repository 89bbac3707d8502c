"""GPU CP-ALS vs the CPU oracle's CP-ALS (standard ALS, Sec. 2.2 context).

FP64: fit trace within 1e-9 of the oracle's, factors and lambda close.
Mixed precision (FP32 / BF16 factors, FP32 MTTKRP, FP64 Cholesky): final
fit within 1e-3 of the FP64 oracle run from the same initial factors.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, encode_dev, factors_dev

pytestmark = pytest.mark.gpu


def test_fp64_uniform_1M_10_iters():
    w = synth.WORKLOADS["uniform3d-1000x1000x1000-1M"]
    spec = w["spec"]
    c, v = synth.make_tensor(spec)
    R = w["R"]
    fs = synth.init_factors(spec.dims, R, seed=0)
    ref = oracle.cpals(c, v, spec.dims, R, 10, 0.0, fs)
    h = encode_dev(c, v, spec.dims, factor_dtype="f64")
    dfs = factors_dev(fs, "f64")
    res = rl.relate_cpals(h, R, 10, 0.0, dfs)
    assert res["iters"] == 10 and res["status"] == 0
    assert np.max(np.abs(res["fit_trace"] - ref["fit_trace"])) <= 1e-9
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-7)
    for f, g in zip(dfs, ref["factors"]):
        assert np.linalg.norm(f.cpu().numpy() - g) <= 1e-6 * np.linalg.norm(g)
    h.close()


def test_planted_rank3_recovered_on_gpu():
    rng = np.random.default_rng(21)
    dims = (12, 10, 8)
    true = [rng.random((d, 3)) + 0.1 for d in dims]
    X = np.einsum("ar,br,cr,r->abc", *true, np.array([3.0, 2.0, 1.0]))
    c = np.stack(np.nonzero(X)).astype(np.uint32)
    v = X[tuple(c)]
    init = [rng.random((d, 3)) for d in dims]
    h = encode_dev(c, v, dims, factor_dtype="f64")
    res = rl.relate_cpals(h, 3, 1000, 0.0, factors_dev(init, "f64"))
    assert res["fit"] > 0.9999
    h.close()


@pytest.mark.parametrize("fdt", ["f32", "bf16"])
def test_mixed_precision_fit_within_1e3(fdt):
    spec = synth.scaled(synth.WORKLOADS["zipf3d-200Kx200Kx5K-50M"]["spec"], 500_000, dims=(20000, 20000, 500))
    c, v = synth.make_tensor(spec)
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float32)
    iters = 8
    ref = oracle.cpals(c, v.astype(np.float64), spec.dims, R, iters, 0.0, [f.astype(np.float64) for f in fs])
    h = encode_dev(c, v, spec.dims, factor_dtype=fdt)
    res = rl.relate_cpals(h, R, iters, 0.0, factors_dev(fs, fdt))
    assert res["iters"] == iters
    assert abs(res["fit"] - ref["fit_trace"][-1]) <= 1e-3, (res["fit"], ref["fit_trace"][-1])
    h.close()


def test_tolerance_stop_and_warm_restart():
    spec = synth.scaled(synth.WORKLOADS["uniform3d-1000x1000x1000-1M"]["spec"], 50_000, dims=(100, 120, 90))
    c, v = synth.make_tensor(spec)
    fs = synth.init_factors(spec.dims, 4, seed=0)
    h = encode_dev(c, v, spec.dims, factor_dtype="f64")
    dfs = factors_dev(fs, "f64")
    r1 = rl.relate_cpals(h, 4, 200, 1e-4, dfs)
    assert r1["iters"] < 200
    # resume from the returned factors (checkpoint = the caller-owned factors)
    r2 = rl.relate_cpals(h, 4, 2, 0.0, dfs)
    assert r2["fit"] >= r1["fit"] - 1e-9
    h.close()


def _graph_run(c, v, dims, R, iters, tol, init, graph):
    s = torch.cuda.Stream()
    h = encode_dev(c, v, dims, factor_dtype="f64", stream=s)
    rl.relate_set_cpals_graph(h, graph)
    dfs = factors_dev(init, "f64")
    torch.cuda.synchronize()
    try:
        res = rl.relate_cpals(h, R, iters, tol, dfs)
    except rl.RelateError as e:
        res = {"error": e.status}
    h.close()
    return res


def test_graph_mode_with_tolerance_stops_like_the_plain_path():
    spec = synth.scaled(synth.WORKLOADS["uniform3d-1000x1000x1000-1M"]["spec"], 50_000, dims=(100, 120, 90))
    c, v = synth.make_tensor(spec)
    init = synth.init_factors(spec.dims, 4, seed=0)
    a = _graph_run(c, v, spec.dims, 4, 200, 1e-4, init, False)
    b = _graph_run(c, v, spec.dims, 4, 200, 1e-4, init, True)
    assert a["iters"] == b["iters"] < 200
    assert np.max(np.abs(a["fit_trace"] - b["fit_trace"])) <= 1e-9


def test_not_positive_definite_reported_in_both_graph_paths():
    """A zero factor makes every V of the other modes zero (even after the
    ridge retry): NOT_PD in the first iteration, with the per-iteration path,
    and with the fixed-count replay that synchronises only at the end."""
    rng = np.random.default_rng(4)
    dims = (40, 30, 20)
    c = np.stack([rng.integers(0, d, 3000) for d in dims]).astype(np.uint32)
    v = rng.random(3000)
    init = [rng.random((d, 4)) for d in dims]
    init[1][:] = 0.0
    for graph in (False, True):
        for tol in (0.0, 1e-6):
            res = _graph_run(c, v, dims, 4, 5, tol, init, graph)
            assert res.get("error") == -6, (graph, tol, res)  # RELATE_ERR_NOT_PD


@pytest.mark.parametrize("graph", [False, True])
def test_ridge_retry_path_matches_the_oracle(graph):
    """A zero column in one initial factor makes the normal-equations matrix
    of every mode singular (a zero pivot): the first Cholesky fails and the
    retry with V + 1e-12 tr(V)/R I succeeds, once per mode and iteration,
    on the GPU as in the oracle. Retry count, fit trace (<= 1e-9), lambda
    and factors are compared; the zero column stays exactly zero."""
    rng = np.random.default_rng(29)
    dims = (300, 250, 200)
    nnz = 20000
    c = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    v = rng.random(nnz)
    R, iters = 6, 4
    init = [rng.random((d, R)) for d in dims]
    init[2][:, 1] = 0.0
    ref = oracle.cpals(c, v, dims, R, iters, 0.0, init)
    assert ref["ridges"] == 3 * iters
    s = torch.cuda.Stream()
    h = encode_dev(c, v, dims, factor_dtype="f64", stream=s)
    rl.relate_set_cpals_graph(h, graph)
    dfs = factors_dev(init, "f64")
    torch.cuda.synchronize()
    res = rl.relate_cpals(h, R, iters, 0.0, dfs)
    h.close()
    assert res["status"] == 0 and res["iters"] == iters
    assert res["ridge_retries"] == ref["ridges"]
    assert np.max(np.abs(res["fit_trace"] - ref["fit_trace"])) <= 1e-9
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-7, atol=0)
    for f, g in zip(dfs, ref["factors"]):
        f = f.cpu().numpy()
        assert np.all(f[:, 1] == 0.0)
        assert np.linalg.norm(f - g) <= 1e-6 * np.linalg.norm(g)


def test_lambda_to_device_memory():
    """relate_cpals writes lambda to a device buffer as well as to a host one."""
    spec = synth.scaled(synth.WORKLOADS["uniform3d-1000x1000x1000-1M"]["spec"], 30_000, dims=(90, 80, 70))
    c, v = synth.make_tensor(spec)
    fs = synth.init_factors(spec.dims, 5, seed=0)
    out = []
    for lam in (None, torch.full((5,), float("nan"), dtype=torch.float64, device=DEV)):
        h = encode_dev(c, v, spec.dims, factor_dtype="f64")
        res = rl.relate_cpals(h, 5, 3, 0.0, factors_dev(fs, "f64"), lam=lam)
        h.close()
        got = res["lam"]
        out.append(got.cpu().numpy() if hasattr(got, "cpu") else got)
    assert np.all(np.isfinite(out[1]))
    np.testing.assert_allclose(out[1], out[0], rtol=1e-10, atol=0)  # atomics order differs between runs


@pytest.mark.parametrize("graph", [0, 1])
def test_fp64_four_modes_with_khatri_rao_pairs(graph):
    """A 4-mode FP64 run whose modes 0 and 1 fuse the same Khatri-Rao pair
    (modes 2 and 3) and mode 2 the pair (1, 3): mode 0 builds the table, mode 1
    reuses it, mode 2 rebuilds it from the updated A_1. Fit trace, lambda and
    factors as the 3-mode FP64 case, in the plain and the graph path."""
    spec = synth.TensorSpec("kr-cpals4d", (6000, 3000, 300, 20), 400_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="uniform", value_dtype="f32", seed=58)
    c, v = synth.make_tensor(spec)
    v = v.astype(np.float64)
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=2)
    ref = oracle.cpals(c, v, spec.dims, R, 6, 0.0, fs)
    h = encode_dev(c, v, spec.dims, factor_dtype="f64")
    assert [rl.relate_get_mode_kr(h, n, R)["kr"] for n in range(4)] == [1, 1, 1, 0]
    rl.relate_set_cpals_graph(h, graph)
    dfs = factors_dev(fs, "f64")
    res = rl.relate_cpals(h, R, 6, 0.0, dfs)
    assert res["iters"] == 6 and res["status"] == 0
    assert np.max(np.abs(res["fit_trace"] - ref["fit_trace"])) <= 1e-9
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-7)
    for f, g in zip(dfs, ref["factors"]):
        assert np.linalg.norm(f.cpu().numpy() - g) <= 1e-6 * np.linalg.norm(g)
    h.close()
