"""The seeded generators: the multithreaded C helper reproduces the numpy
definitions exactly, draws are deterministic, coordinates are distinct and
in range."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name,nnz", [("zipf3d-200Kx200Kx5K-50M", 200_000),
                                      ("zipf4d-5Mx1Mx100Kx24-150M", 100_000),
                                      ("zipf5d-10Mx10Mx1Mx1Kx100-100M", 100_000),
                                      ("uniform3d-1000x1000x1000-1M", 100_000)])
@pytest.mark.parametrize("shuffle", [False, True])
def test_c_helper_matches_numpy(name, nnz, shuffle):
    spec = synth.scaled(synth.WORKLOADS[name]["spec"], nnz)
    spec.shuffle = shuffle
    a = synth.make_coords(spec, use_c=True)
    b = synth.make_coords(spec, use_c=False)
    assert np.array_equal(a, b)
    assert a.shape == (len(spec.dims), nnz)
    for n, I in enumerate(spec.dims):
        assert int(a[n].max()) < I
    lin = np.zeros(nnz, dtype=object)
    for n, I in enumerate(spec.dims):
        lin = lin * int(I) + a[n].astype(object)
    assert len(set(lin.tolist())) == nnz


def test_values_and_factors_deterministic():
    spec = synth.scaled(synth.WORKLOADS["zipf3d-200Kx200Kx5K-50M"]["spec"], 1000)
    v1, v2 = synth.make_values(spec), synth.make_values(spec)
    assert v1.dtype == np.float32 and np.array_equal(v1, v2) and (v1 > 0).all()
    f = synth.init_factors((10, 20), 4)
    assert f[0].shape == (10, 4) and f[1].shape == (20, 4)
    assert (f[0] > 0).all() and (f[0] <= 1).all()
    # factors drawn in order (mode, row, column) from one stream
    g = synth.init_factors((10,), 4)
    assert np.array_equal(f[0], g[0])
