"""Sharded CP-ALS through the library (relate_encode shard_rank / shard_count,
relate_set_reduce_hook) on one GPU.

Two shard handles of one tensor run relate_cpals on two host threads; their
reduce hook sums the two partial buffers in process (each thread synchronises
its stream, meets the other at a host barrier, adds the other shard's buffer
with a torch kernel of its own and meets it again): no kernel waits for
another, the host does the meeting. Every mode's partial MTTKRP and ||X||^2
are summed as a multi-GPU run would sum them with NCCL. The FP64 fit trace,
lambda and factors must equal the unsharded run's within 1e-9 / 1e-7, and the
shards must tile the sorted stream (relate_get_stats: shard_lo, nnz).
"""
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from paper_2509_00280_gb300 import shard
from gpu_util import DEV, factors_dev

pytestmark = pytest.mark.gpu


def _tensor():
    spec = synth.TensorSpec("shard-gpu", (3000, 2000, 400, 24), 600_000, (("zipf", 1.1),) * 3 + (("uniform",),),
                            values="uniform", value_dtype="f32", seed=71)
    return spec, *synth.make_tensor(spec)


class InProcessReduce:
    """The all-reduce of `world` host threads of this process."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world)
        self.bufs = [None] * world

    def hook(self, rank):
        def fn(buf, count, dtype, stream):
            st = torch.cuda.ExternalStream(stream)
            st.synchronize()
            t = shard.device_view(buf, count, dtype)
            self.bufs[rank] = t
            self.bar.wait(timeout=120)
            total = sum(b.clone() for b in self.bufs)  # every thread forms the same sum
            self.bar.wait(timeout=120)
            t.copy_(total)
            torch.cuda.current_stream().synchronize()
            self.bar.wait(timeout=120)
            return 0
        return fn


@pytest.mark.parametrize("fdt", ["f64", "f32"])
def test_two_shards_on_threads_match_the_unsharded_run(fdt):
    spec, c, v = _tensor()
    R, iters = 16, 5
    init = synth.init_factors(spec.dims, R, seed=0)
    dc, dv = torch.from_numpy(c).to(DEV), torch.from_numpy(v).to(DEV)
    s0 = torch.cuda.Stream()
    h = rl.relate_encode(dc, dv, spec.dims, factor_dtype=fdt, stream=s0)
    ref = rl.relate_cpals(h, R, iters, 0.0, factors_dev(init, fdt))
    h.close()

    world = 2
    red = InProcessReduce(world)
    out = [None] * world
    errs = []

    def run(rank):
        try:
            torch.cuda.set_device(DEV)
            st = torch.cuda.Stream()
            hs = shard.sharded_encode(dc, dv, spec.dims, rank, world, factor_dtype=fdt, stream=st)
            stats = rl.relate_get_stats(hs)
            f = factors_dev(init, fdt)
            rl.relate_set_reduce_hook(hs, red.hook(rank))
            res = rl.relate_cpals(hs, R, iters, 0.0, f)
            hs.close()
            out[rank] = (stats, res, [x.double().cpu().numpy() for x in f])
        except BaseException as e:  # reported by the main thread
            errs.append(e)
            red.bar.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errs, errs
    (s0_, r0, f0), (s1_, r1, f1) = out
    assert s0_["nnz_total"] == s1_["nnz_total"] == spec.nnz
    assert s0_["shard_lo"] == 0 and s1_["shard_lo"] == s0_["nnz"] and s0_["nnz"] + s1_["nnz"] == spec.nnz
    tol = 1e-9 if fdt == "f64" else 1e-5
    for r in (r0, r1):
        assert r["iters"] == iters and r["status"] == 0
        assert np.max(np.abs(r["fit_trace"] - ref["fit_trace"])) <= tol
        np.testing.assert_allclose(r["lam"], ref["lam"], rtol=1e-7 if fdt == "f64" else 1e-3)
    for a, b in zip(f0, f1):  # replicated updates from the same sums
        assert np.max(np.abs(a - b)) <= (1e-12 if fdt == "f64" else 1e-6)


def test_one_shard_is_the_unsharded_encoding():
    spec, c, v = _tensor()
    dc, dv = torch.from_numpy(c).to(DEV), torch.from_numpy(v).to(DEV)
    a = rl.relate_encode(dc, dv, spec.dims)
    b = shard.sharded_encode(dc, dv, spec.dims, 0, 1)
    sa, sb = rl.relate_get_stats(a), rl.relate_get_stats(b)
    for k in ("nnz", "partitions", "runs", "distinct", "maxcount", "bit_order"):
        assert sa[k] == sb[k]
    assert sb["nnz_total"] == spec.nnz and sb["shard_lo"] == 0
    a.close()
    b.close()


def test_shard_keeps_its_slice_of_the_sorted_stream():
    spec, c, v = _tensor()
    dc, dv = torch.from_numpy(c).to(DEV), torch.from_numpy(v).to(DEV)
    enc = oracle.encode_full(c, v, spec.dims)
    for rank, world in ((0, 3), (1, 3), (2, 3)):
        h = shard.sharded_encode(dc, dv, spec.dims, rank, world)
        lo, hi = rl.relate_shard_range(spec.nnz, rank, world)
        st = rl.relate_get_stats(h)
        assert (st["shard_lo"], st["nnz"]) == (lo, hi - lo)
        perm = torch.empty(hi - lo, dtype=torch.int32, device=DEV)
        rl.relate_decode(h, perm_out=perm)
        torch.cuda.synchronize()
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), enc["perm"][lo:hi])
        h.close()
