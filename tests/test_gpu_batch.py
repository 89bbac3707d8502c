"""The batched MTTKRP (one persistent launch over the tiles of several
problems) and the lockstep CP-ALS of several problems, against the oracle and
against each problem alone (Sec. 2.2, Fig. 2 for the MTTKRP; the standard ALS
for CP-ALS).

Tolerances: MTTKRP relative Frobenius error FP64 <= 1e-12, FP32 <= 1e-5
against the oracle; CP-ALS fit trace FP64 within 1e-9 of the oracle's and of
the problem alone; FP32 fits within 1e-6 of the problem alone (the same
arithmetic, another order of atomic additions).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, TORCH_DT, encode_dev, factors_dev, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _problem(i, N, nnz, dims, fdt, R, seed):
    spec = synth.TensorSpec(f"batch-{i}", dims, nnz, (("zipf", 1.2),) * N, values="uniform",
                            value_dtype="f64" if fdt == "f64" else "f32", seed=seed, distinct="once")
    c, v = synth.make_tensor(spec)
    fs = synth.init_factors(dims, R, seed=seed + 100)
    if fdt == "f32":
        fs = [f.astype(np.float32).astype(np.float64) for f in fs]
    return spec, c, v, fs


PROBLEMS = [(3, 40_000, (300, 200, 150), 8), (3, 120_000, (2000, 900, 60), 16), (3, 9_000, (100, 120, 90), 32),
            (4, 60_000, (500, 400, 30, 20), 16), (5, 30_000, (100, 90, 80, 12, 7), 8), (3, 70_000, (800, 600, 50), 16)]


@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_mttkrp_batch_matches_the_oracle_and_single_launches(fdt):
    probs = [_problem(i, *p[:3], fdt, p[3], 60 + i) for i, p in enumerate(PROBLEMS)]
    hs, dfs, items, refs, alone = [], [], [], [], []
    acc = torch.float64 if fdt == "f64" else torch.float32
    for (spec, c, v, fs), (N, _, dims, R) in zip(probs, PROBLEMS):
        h = encode_dev(c, v, dims, factor_dtype=fdt)
        d = factors_dev(fs, fdt)
        hs.append(h)
        dfs.append(d)
        for n in range(N):
            out = torch.full((dims[n], R), float("nan"), dtype=acc, device=DEV)
            items.append((h, n, d, R, out))
            refs.append(oracle.mttkrp(c, v.astype(np.float64), dims, n, fs))
            one = torch.empty_like(out)
            rl.relate_mttkrp(h, n, d, R, one)
            alone.append(one)
    # a misaligned item (factor one element off 16 bytes) takes the single-launch path
    spec, c, v, fs = probs[1]
    N, _, dims, R = PROBLEMS[1]
    mis = []
    for f in fs:
        flat = torch.zeros(f.size + 1, dtype=TORCH_DT[fdt], device=DEV)
        view = flat[1:].view(f.shape)
        view.copy_(torch.from_numpy(f).to(DEV).to(TORCH_DT[fdt]))
        mis.append(view)
    out_mis = torch.empty((dims[0], R), dtype=acc, device=DEV)
    items.append((hs[1], 0, mis, R, out_mis))
    refs.append(oracle.mttkrp(c, v.astype(np.float64), dims, 0, fs))
    alone.append(None)
    rl.relate_mttkrp_batch(items)
    torch.cuda.synchronize()
    for (h, n, d, R, out), ref, one in zip(items, refs, alone):
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert rel_fro(got, ref) <= TOL[fdt], (fdt, n, R)
        if one is not None:
            assert rel_fro(got, one.cpu().numpy().astype(np.float64)) <= TOL[fdt]
    for h in hs:
        rl.relate_sync_status(h)
        h.close()


def _cpals_alone(spec, c, v, dims, R, fdt, iters, tol, fs):
    s = torch.cuda.Stream()
    h = encode_dev(c, v, dims, factor_dtype=fdt, stream=s)
    res = rl.relate_cpals(h, R, iters, tol, factors_dev(fs, fdt))
    h.close()
    return res


def test_cpals_batch_fp64_matches_alone_and_the_oracle():
    probs = [_problem(i, *p[:3], "f64", p[3], 80 + i) for i, p in enumerate(PROBLEMS)]
    s = torch.cuda.Stream()
    hs, facs = [], []
    for (spec, c, v, fs), (N, _, dims, R) in zip(probs, PROBLEMS):
        hs.append(encode_dev(c, v, dims, factor_dtype="f64", stream=s))
        facs.append(factors_dev(fs, "f64"))
    Rs = [p[3] for p in PROBLEMS]
    res, rc = rl.relate_cpals_batch(hs, Rs, 40, 1e-4, facs, s)
    assert rc == 0
    iters_seen = set()
    for r, (spec, c, v, fs), (N, _, dims, R) in zip(res, probs, PROBLEMS):
        alone = _cpals_alone(spec, c, v, dims, R, "f64", 40, 1e-4, fs)
        ref = oracle.cpals(c, v, dims, R, 40, 1e-4, fs)
        assert r["status"] == 0
        assert r["iters"] == alone["iters"] == ref["iters"]
        assert np.max(np.abs(r["fit_trace"] - alone["fit_trace"])) <= 1e-9
        assert np.max(np.abs(r["fit_trace"] - ref["fit_trace"])) <= 1e-9
        np.testing.assert_allclose(r["lam"], ref["lam"], rtol=1e-7)
        iters_seen.add(r["iters"])
    assert len(iters_seen) > 1  # problems stopped at different iterations (graph re-captured)
    for h in hs:
        h.close()


def test_cpals_batch_fp32_same_alone_and_in_the_mix():
    probs = [_problem(i, *p[:3], "f32", p[3], 90 + i) for i, p in enumerate(PROBLEMS)]
    s = torch.cuda.Stream()

    def run(idx):
        hs = [encode_dev(probs[i][1], probs[i][2], PROBLEMS[i][2], factor_dtype="f32", stream=s) for i in idx]
        facs = [factors_dev(probs[i][3], "f32") for i in idx]
        res, rc = rl.relate_cpals_batch(hs, [PROBLEMS[i][3] for i in idx], 12, 0.0, facs, s)
        for h in hs:
            h.close()
        assert rc == 0
        return res

    mix = run(list(range(len(PROBLEMS))))
    for i in range(len(PROBLEMS)):
        one = run([i])[0]
        assert one["iters"] == mix[i]["iters"] == 12
        assert np.max(np.abs(one["fit_trace"] - mix[i]["fit_trace"])) <= 1e-6, i


def test_cpals_batch_resume_with_prev_fit():
    """Two calls of 5 iterations, the second resumed with the first's last fit,
    follow the one-call run (the Grams are formed again from the factors, so
    the traces agree up to rounding)."""
    spec, c, v, fs = _problem(0, *PROBLEMS[1][:3], "f64", PROBLEMS[1][3], 95)
    dims, R = PROBLEMS[1][2], PROBLEMS[1][3]
    s = torch.cuda.Stream()
    h = encode_dev(c, v, dims, factor_dtype="f64", stream=s)
    f = factors_dev(fs, "f64")
    a, _ = rl.relate_cpals_batch([h], [R], 5, 0.0, [f], s)
    b, _ = rl.relate_cpals_batch([h], [R], 5, 0.0, [f], s, prev_fit=[a[0]["fit"]])
    h.close()
    one = _cpals_alone(spec, c, v, dims, R, "f64", 10, 0.0, fs)
    both = np.concatenate([a[0]["fit_trace"], b[0]["fit_trace"]])
    assert np.max(np.abs(both - one["fit_trace"])) <= 1e-9


def test_cpals_batch_reports_an_injected_timeout(monkeypatch):
    spec, c, v, fs = _problem(0, *PROBLEMS[0][:3], "f32", PROBLEMS[0][3], 96)
    dims, R = PROBLEMS[0][2], PROBLEMS[0][3]
    s = torch.cuda.Stream()
    h = encode_dev(c, v, dims, factor_dtype="f32", stream=s)
    f = factors_dev(fs, "f32")
    monkeypatch.setenv("RELATE_FAULT", "timeout")
    res, rc = rl.relate_cpals_batch([h], [R], 3, 0.0, [f], s)
    assert rc == -7 and res[0]["status"] == -7
    monkeypatch.delenv("RELATE_FAULT")
    res, rc = rl.relate_cpals_batch([h], [R], 3, 0.0, [factors_dev(fs, "f32")], s)
    assert rc == 0 and res[0]["iters"] == 3
    h.close()
