"""Sharded CP-ALS across processes, on the CPU with gloo (world size 2).

The nonzero stream shards naturally: each rank keeps the contiguous
equal-nnz slice of the sorted stream that the library's relate_shard_range
assigns it, computes its partial mode-n MTTKRP, and the partials are summed
by the reduction the library calls after every mode (shard.host_reduce_hook,
the host-memory form of the hook relate_cpals calls through
relate_set_reduce_hook), as is ||X||^2 once; the Grams, normal equations and
fit are replicated. The per-rank compute is the CPU oracle's (no GPU here),
following the library's protocol step by step; the sharded fit trace must
equal the unsharded oracle CP-ALS within 1e-9 and every rank must end with
the same factors.
"""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
import paper_2509_00280_gb300 as rl
from paper_2509_00280_gb300 import shard

SPEC = synth.TensorSpec("shard", (60, 45, 30), 20000, (("zipf", 1.1),) * 3, values="uniform",
                        value_dtype="f64", seed=5)
R, ITERS = 6, 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _reduce(hook, arr):
    """Calls the hook as the library does: (device or host address, count, dtype, stream)."""
    a = np.ascontiguousarray(arr)
    rc = hook(a.ctypes.data, a.size, rl.RELATE_F64, None)
    assert rc == 0
    return a


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, v = synth.make_tensor(SPEC)
        enc = oracle.encode_full(c, v, SPEC.dims, S=512)
        lo, hi = rl.relate_shard_range(c.shape[1], rank, world)
        cs, vs = np.ascontiguousarray(enc["coords"][:, lo:hi]), enc["vals"][lo:hi]
        hook = shard.host_reduce_hook()
        fs = synth.init_factors(SPEC.dims, R, seed=0)
        N = len(SPEC.dims)
        normX2 = _reduce(hook, np.array([float(np.sum(vs * vs))]))[0]
        G = [oracle.gram(f) for f in fs]
        trace = []
        for _ in range(ITERS):
            for n in range(N):
                M = _reduce(hook, oracle.mttkrp(cs, vs, SPEC.dims, n, fs))  # partial MTTKRP, then summed
                V = np.ones((R, R))
                for k in range(N):
                    if k != n:
                        V *= G[k]
                A = oracle.solve_rows(M, V)
                lam = np.linalg.norm(A, axis=0)
                fs[n] = A / lam
                G[n] = oracle.gram(fs[n])
            H = np.ones((R, R))
            for k in range(N):
                H *= G[k]
            inner = float(np.sum(lam * np.sum(M * fs[N - 1], axis=0)))
            res2 = normX2 + lam @ H @ lam - 2.0 * inner
            trace.append(1.0 - np.sqrt(max(res2, 0.0)) / np.sqrt(normX2))
        q.put((rank, (lo, hi), np.array(trace), [f.copy() for f in fs]))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_sharded_cpals_matches_single_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(world):
        rank, rng, trace, fs = q.get(timeout=240)
        results[rank] = (rng, trace, fs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c, v = synth.make_tensor(SPEC)
    # the library's shards tile the stream: contiguous, disjoint, equal within one nonzero
    assert results[0][0][0] == 0 and results[0][0][1] == results[1][0][0] and results[1][0][1] == c.shape[1]
    sizes = [hi - lo for lo, hi in (results[0][0], results[1][0])]
    assert max(sizes) - min(sizes) <= 1
    ref = oracle.cpals(c, v, SPEC.dims, R, ITERS, 0.0, synth.init_factors(SPEC.dims, R, seed=0))
    for r in range(world):
        assert np.max(np.abs(results[r][1] - ref["fit_trace"])) <= 1e-9
        for a, b in zip(results[r][2], ref["factors"]):
            np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-10)
    for a, b in zip(results[0][2], results[1][2]):
        assert np.array_equal(a, b)  # replicated: bit-identical on every rank


def test_shard_range_tiles_the_stream():
    for nnz in (0, 1, 7, 1000, 2**33 + 5):
        for world in (1, 2, 3, 8):
            bounds = [rl.relate_shard_range(nnz, r, world) for r in range(world)]
            assert bounds[0][0] == 0 and bounds[-1][1] == nnz
            assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in bounds]
            assert max(sizes) - min(sizes) <= 1


def test_host_reduce_hook_is_the_libraries_callback_type():
    """The reduction is handed to the library as a relate_reduce_fn."""
    called = []

    def fn(buf, count, dtype, stream):
        called.append((count, dtype))
        return 0

    cb = rl.relate.REDUCE_FN(lambda b, n, d, s, u: fn(b, n, d, s))
    x = np.zeros(3)
    assert cb(x.ctypes.data, 3, rl.RELATE_F64, None, None) == 0
    assert called == [(3, rl.RELATE_F64)]
    assert ctypes.cast(cb, ctypes.c_void_p).value
