"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/relate.h; host-side argument checks fail cleanly. No
compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def relate_lib():
    from paper_2509_00280_gb300 import build_lib
    build_lib.build()
    import paper_2509_00280_gb300 as rl
    return rl


def _declared():
    txt = open(os.path.join(ROOT, "include", "relate.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(relate_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(relate_lib):
    names = _declared()
    assert "relate_encode" in names and "relate_mttkrp" in names and "relate_cpals" in names
    so = ctypes.CDLL(relate_lib.library_path())
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_status_strings_and_version(relate_lib):
    assert relate_lib.relate_status_string(0) == "ok"
    for s in range(-1, -10, -1):
        assert relate_lib.relate_status_string(s) not in ("ok", "unknown status")
    assert "sm_103a" in relate_lib.relate_version()


def test_host_side_validation_without_gpu(relate_lib):
    L = relate_lib.lib()
    out = ctypes.c_void_p(0)
    dims = np.array([4, 8, 2], dtype=np.uint64)
    # nmodes out of range
    assert L.relate_encode(None, None, dims.ctypes.data, 1, 0, None, ctypes.byref(out)) == -1
    assert L.relate_encode(None, None, dims.ctypes.data, 9, 0, None, ctypes.byref(out)) == -1
    # NULL out
    assert L.relate_encode(None, None, dims.ctypes.data, 3, 0, None, None) == -1
    # l(p) > 128 bits
    wide = np.array([2 ** 32] * 5, dtype=np.uint64)
    assert L.relate_encode(None, None, wide.ctypes.data, 5, 0, None, ctypes.byref(out)) == -3
    # bad bit order (mode 0 needs 2 bits)
    p = relate_lib.relate.Params()
    L.relate_params_default(ctypes.byref(p))
    order = np.array([2, 0, 1, 1, 1, 1], dtype=np.int8)
    p.bit_order = order.ctypes.data
    p.bit_order_len = 6
    assert L.relate_encode(None, None, dims.ctypes.data, 3, 0, ctypes.byref(p), ctypes.byref(out)) == -2
    # NULL handle everywhere
    assert L.relate_mttkrp(None, 0, None, 16, None, None) == -1
    assert L.relate_cpals(None, 16, 1, 0.0, None, None, None) == -1
    assert L.relate_get_stats(None, None) == -1
    assert "NULL" in relate_lib.relate_last_error()
    L.relate_free(None)  # no-op


def test_params_struct_layout_matches_header(relate_lib):
    """The ctypes mirror of relate_params_t round-trips through the C default
    initialiser (a layout mismatch would scramble these fields)."""
    p = relate_lib.relate.Params()
    relate_lib.lib().relate_params_default(ctypes.byref(p))
    assert p.partition_size == 0 and list(p.conflict) == [0] * 8
    assert (p.val_dtype, p.factor_dtype, p.acc_dtype) == (1, 1, 1)
    assert p.coords_on_device == 0 and p.smem_budget == 0
