"""Sharded MTTKRP / CP-ALS step arithmetic across ranks, on the CPU with gloo.

The nonzero stream shards naturally: each rank takes a contiguous equal-nnz
slice of the encoded (position-ordered) stream, computes the partial mode-n
MTTKRP of its slice, and the partials are summed across ranks (one all-reduce
per mode); the Grams are tiny (R x R) and replicated. This checks, with two
gloo ranks and the CPU oracle as the per-rank compute, that the sum of the
shard partials equals the unsharded MTTKRP and that a sharded ALS sweep
reproduces the single-rank factors. Only the arithmetic of the exchange is
tested here: every run of this library uses one GPU per process.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard(n, world, rank):
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = synth.TensorSpec("shard", (60, 45, 30), 20000, (("zipf", 1.1),) * 3, values="uniform",
                                value_dtype="f64", seed=5)
        c, v = synth.make_tensor(spec)
        enc = oracle.encode_full(c, v, spec.dims, S=512)
        cs, vs = enc["coords"], enc["vals"]
        lo, hi = _shard(cs.shape[1], world, rank)
        R = 6
        fs = synth.init_factors(spec.dims, R, seed=0)
        out = []
        # one sharded ALS sweep: partial MTTKRP per rank, all-reduce, replicated solve
        for n in range(3):
            part = oracle.mttkrp(np.ascontiguousarray(cs[:, lo:hi]), vs[lo:hi], spec.dims, n, fs)
            t = torch.from_numpy(part)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            M = t.numpy()
            V = np.ones((R, R))
            for k in range(3):
                if k != n:
                    V *= oracle.gram(fs[k])
            A = oracle.solve_rows(M, V)
            lam = np.linalg.norm(A, axis=0)
            fs[n] = A / lam
            out.append(M.copy())
        q.put((rank, out, [f.copy() for f in fs]))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_shards_reproduce_single_rank_sweep():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(world):
        rank, Ms, fs = q.get(timeout=240)
        results[rank] = (Ms, fs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # single-rank reference sweep
    spec = synth.TensorSpec("shard", (60, 45, 30), 20000, (("zipf", 1.1),) * 3, values="uniform",
                            value_dtype="f64", seed=5)
    c, v = synth.make_tensor(spec)
    R = 6
    fs = synth.init_factors(spec.dims, R, seed=0)
    for n in range(3):
        M = oracle.mttkrp(c, v, spec.dims, n, fs)
        V = np.ones((R, R))
        for k in range(3):
            if k != n:
                V *= oracle.gram(fs[k])
        A = oracle.solve_rows(M, V)
        fs[n] = A / np.linalg.norm(A, axis=0)
        for r in range(world):
            np.testing.assert_allclose(results[r][0][n], M, rtol=1e-12, atol=1e-12)
    for r in range(world):
        for a, b in zip(results[r][1], fs):
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)
