"""Autotuner on the GPU: the tuned encoding computes the same MTTKRP as the
oracle, and it is never slower than the ALTO baseline it is scored against."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from paper_2509_00280_gb300 import tune
from gpu_util import DEV, encode_dev, factors_dev, mttkrp_dev, rel_fro

pytestmark = pytest.mark.gpu


def test_tuned_encoding_is_correct_and_not_slower():
    spec = synth.scaled(synth.WORKLOADS["zipf4d-5Mx1Mx100Kx24-150M"]["spec"], 400_000)
    c, v = synth.make_tensor(spec)
    R = 16
    fs = synth.init_factors(spec.dims, R, seed=0, dtype=np.float32)
    dfs = factors_dev(fs, "f32")
    ev = tune.gpu_evaluator(torch.from_numpy(c).to(DEV), torch.from_numpy(v).to(DEV), spec.dims, R, "f32", dfs,
                            reps=2)
    res = tune.tune(spec.dims, ev, partition_sizes=(4096, 2048), max_evals=10, patience=6)
    assert res.best.seconds <= res.baseline.seconds
    assert oracle.check_order(spec.dims, res.best.order)
    h = encode_dev(c, v, spec.dims, bit_order=np.array(res.best.order, dtype=np.int8),
                   partition_size=res.best.partition_size, factor_dtype="f32")
    for n, strat in enumerate(res.best.strategies):
        rl.relate_set_conflict(h, n, strat)
    for n in range(4):
        ref = oracle.mttkrp(c, v.astype(np.float64), spec.dims, n, [f.astype(np.float64) for f in fs])
        assert rel_fro(mttkrp_dev(h, n, dfs, R), ref) <= 1e-5
    h.close()
