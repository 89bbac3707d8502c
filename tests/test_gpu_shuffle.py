"""Invariance of the MTTKRP under label shuffling (the paper's shuffled
workloads, Sec. 4.1.3: every mode's labels relabelled by a seeded
permutation), on the GPU.

With pi_n the label permutation of mode n, the shuffled tensor holds the
nonzero (pi_0(i_0), ..., pi_{N-1}(i_{N-1}), v) for every original nonzero, so
with factors relabelled the same way (A'_k(pi_k(i), :) = A_k(i, :)) the
mode-n MTTKRP satisfies M'(pi_n(i), :) = M(i, :) (Sec. 2.2, Fig. 2). The two
tensors encode to different orders, tiles and strategies; their outputs are
compared element by element after relabelling, at the MTTKRP tolerances
(FP64 1e-12, FP32 1e-5 relative Frobenius).
"""
import dataclasses

import numpy as np
import pytest
import torch

import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, TORCH_DT, encode_dev, rel_fro

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("name,nnz", [("zipf3d-200Kx200Kx5K-50M", 2_000_000), ("zipf4d-5Mx1Mx100Kx24-150M", 3_000_000)])
@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_shuffled_labels_give_the_relabelled_mttkrp(name, nnz, fdt):
    w = synth.WORKLOADS[name]
    base = synth.scaled(w["spec"], nnz)
    shuf = dataclasses.replace(base, shuffle=True)
    c, v = synth.make_tensor(base)
    cs, vs = synth.make_tensor(shuf)
    N = len(base.dims)
    pis = [synth.label_permutation(base.seed, n, int(base.dims[n])) for n in range(N)]
    # the generator relabels the same draws: the shuffled tensor is pi(original)
    assert np.array_equal(vs, v)
    for n in range(N):
        assert np.array_equal(cs[n], pis[n][c[n]])
    R = 32
    fs = synth.init_factors(base.dims, R, seed=0)
    fs_shuf = []
    for n in range(N):
        f = np.empty_like(fs[n])
        f[pis[n]] = fs[n]
        fs_shuf.append(f)
    ha = encode_dev(c, v, base.dims, factor_dtype=fdt)
    hb = encode_dev(cs, vs, base.dims, factor_dtype=fdt)
    da = [torch.from_numpy(f).to(DEV).to(TORCH_DT[fdt]).contiguous() for f in fs]
    db = [torch.from_numpy(f).to(DEV).to(TORCH_DT[fdt]).contiguous() for f in fs_shuf]
    acc = torch.float64 if fdt == "f64" else torch.float32
    for n in range(N):
        oa = torch.empty((base.dims[n], R), dtype=acc, device=DEV)
        ob = torch.empty_like(oa)
        rl.relate_mttkrp(ha, n, da, R, oa)
        rl.relate_mttkrp(hb, n, db, R, ob)
        torch.cuda.synchronize()
        relabelled = ob.cpu().numpy().astype(np.float64)[pis[n]]
        assert rel_fro(relabelled, oa.cpu().numpy().astype(np.float64)) <= TOL[fdt], (name, fdt, n)
    ha.close()
    hb.close()
