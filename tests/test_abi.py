"""The C-ABI library loads and exports every declared entry point; host-side argument
validation runs without a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pch():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1305_1293_gb300 import pch as p
    return p


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pch.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pch_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pch):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(pch.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_struct_sizes_match_header(pch):
    assert ctypes.sizeof(pch.Source) == 40
    assert ctypes.sizeof(pch.Options) == 48
    assert ctypes.sizeof(pch.Stats) == 208
    assert pch.CONTOUR_DTYPE.itemsize == 32             # pch_contour_segment: 4 int32 + 2 double


def test_mlp_shape(pch):
    assert pch.mlp_num_features() == 24
    assert pch.mlp_num_params() == 64 * 24 + 64 + 2 * (64 * 64 + 64) + 64 + 1


@pytest.mark.parametrize("case", ["oob_index", "negative_index", "nan_coord", "too_few"])
def test_create_mesh_rejects_bad_input_on_host(pch, case):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.float64)
    f = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    if case == "oob_index":
        f[1, 1] = 7
    elif case == "negative_index":
        f[0, 0] = -1
    elif case == "nan_coord":
        v[2, 1] = np.nan
    else:
        v = v[:2]
    with pytest.raises(pch.PchError) as e:
        pch.Mesh(v, f)
    assert e.value.status == pch.PCH_ERR_INVALID_ARG
    assert pch.lib.pch_last_error().decode() != ""


def test_null_arguments(pch):
    assert pch.lib.pch_create_mesh(None, 3, None, 1, None) == pch.PCH_ERR_INVALID_ARG
    assert pch.lib.pch_solve(None, None, None, None, None) == pch.PCH_ERR_INVALID_ARG
    assert pch.lib.pch_mesh_info(None, None, None, None, None) == pch.PCH_ERR_INVALID_ARG
    pch.lib.pch_destroy(None)   # no-op
    bad = np.zeros(10, dtype=np.float32)
    assert pch.lib.pch_mlp_set_weights(bad.ctypes.data, 10) == pch.PCH_ERR_INVALID_ARG
