"""GPU encoder vs the CPU oracle: bit-exact positions, permutation, decoded
coordinates, values, partition bounds and fiber statistics (Sec. 3.3)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2509_00280_gb300 as rl
from gpu_util import DEV, decode_all, encode_dev, to_dev

pytestmark = pytest.mark.gpu


def _check_encoding(coords, vals, dims, order=None, S=4096, host_inputs=False):
    N, nnz = coords.shape
    vdt = "f64" if vals.dtype == np.float64 else "f32"
    if host_inputs:
        h = rl.relate_encode(coords, vals, dims, bit_order=order, partition_size=S)
    else:
        h = encode_dev(coords, vals, dims, bit_order=order, partition_size=S)
    ref = oracle.encode_full(coords, vals, dims, order=order, S=S)
    st = rl.relate_get_stats(h)
    assert st["lp"] == oracle.bit_budget(dims)[1]
    assert st["bit_order"] == [int(x) for x in ref["order"]]
    c, v, p, klo, khi = decode_all(h, nnz, N, vdt)
    assert np.array_equal(p, ref["perm"])
    assert np.array_equal(klo, ref["key_lo"]) and np.array_equal(khi, ref["key_hi"])
    assert np.array_equal(c, ref["coords"])
    assert np.array_equal(v, ref["vals"])
    P = st["partitions"]
    assert P == (nnz + S - 1) // S
    if P:
        lo = torch.empty((P, N), dtype=torch.int32, device=DEV)
        hi = torch.empty((P, N), dtype=torch.int32, device=DEV)
        rl.relate_get_partitions(h, lo, hi)
        torch.cuda.synchronize()
        assert np.array_equal(lo.cpu().numpy().view(np.uint32), ref["part_lo"])
        assert np.array_equal(hi.cpu().numpy().view(np.uint32), ref["part_hi"])
    assert st["runs"] == ref["runs"].tolist()
    assert st["distinct"] == ref["distinct"].tolist()
    assert st["maxcount"] == ref["maxcount"].tolist()
    h.close()


def test_worked_example_all_60_orders():
    dims = (4, 8, 2)
    cells = np.array(list(itertools.product(range(4), range(8), range(2))), dtype=np.uint32).T.copy()
    vals = np.arange(64, dtype=np.float32)
    lbits, _ = oracle.bit_budget(dims)
    base = [n for n, l in enumerate(lbits) for _ in range(l)]
    for order in sorted(set(itertools.permutations(base))):
        _check_encoding(cells, vals, dims, order=np.array(order, dtype=np.int8), S=7)


@pytest.mark.parametrize("name,nnz,S", [
    ("uniform3d-1000x1000x1000-1M", 1_000_000, 4096),   # full size, 30-bit keys
    ("zipf3d-200Kx200Kx5K-50M", 300_000, 4096),          # 49-bit keys
    ("zipf4d-5Mx1Mx100Kx24-150M", 200_000, 1000),        # 65-bit keys
    ("zipf5d-10Mx10Mx1Mx1Kx100-100M", 200_000, 777),     # 85-bit keys
])
def test_workload_shapes(name, nnz, S):
    spec = synth.scaled(synth.WORKLOADS[name]["spec"], nnz)
    coords, vals = synth.make_tensor(spec)
    _check_encoding(coords, vals, spec.dims, S=S)


def test_custom_orders_ragged_tail_and_duplicates():
    rng = np.random.default_rng(5)
    dims = (37, 1000, 3, 1, 70000)
    coords = np.stack([rng.integers(0, d, 12345) for d in dims]).astype(np.uint32)
    coords[:, 100:200] = coords[:, 0:1]  # duplicates: stable order must keep input order
    vals = rng.random(12345)
    order = list(oracle.alto_order(dims))
    rng.shuffle(order)
    _check_encoding(coords, vals, dims, order=np.array(order, dtype=np.int8), S=999)
    mode_high = sorted(order, key=lambda m: m == 4)  # mode 4's bits on top
    _check_encoding(coords, vals, dims, order=np.array(mode_high, dtype=np.int8), S=4096, host_inputs=True)


def test_tiny_and_empty():
    dims = (5, 6)
    c = np.array([[4], [5]], dtype=np.uint32)
    _check_encoding(c, np.array([2.5], dtype=np.float32), dims, S=1)
    h = encode_dev(np.zeros((3, 0), dtype=np.uint32), np.zeros(0, dtype=np.float32), (3, 4, 5))
    st = rl.relate_get_stats(h)
    assert st["nnz"] == 0 and st["partitions"] == 0
    out = torch.full((3, 4), 7.0, dtype=torch.float32, device=DEV)
    fs = [torch.ones((d, 4), dtype=torch.float32, device=DEV) for d in (3, 4, 5)]
    rl.relate_mttkrp(h, 0, fs, 4, out)
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0
    h.close()


def test_errors_reported():
    dims = (4, 8, 2)
    c = np.array([[3, 1], [7, 8], [1, 0]], dtype=np.uint32)  # i_1 = 8 >= 8
    with pytest.raises(rl.RelateError) as ei:
        encode_dev(c, np.ones(2, dtype=np.float32), dims)
    assert ei.value.status == -4
    with pytest.raises(rl.RelateError) as ei:
        encode_dev(c[:, :1], np.ones(1, dtype=np.float32), dims, bit_order=np.array([0, 0, 1, 1, 1, 1], np.int8))
    assert ei.value.status == -2
    # the context is still usable after the errors
    _check_encoding(c[:, :1].copy(), np.ones(1, dtype=np.float32), dims)
