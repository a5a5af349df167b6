"""The C ABI without a GPU: the library builds and loads, exports every entry
point include/lbm.h declares, and its host-side model tables (its own Formula 5
solve) agree with the oracle's; invalid arguments fail before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle.model import get_model


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "lbm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    names = declared_entry_points()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lbm):
    assert sorted(lbm.SYMBOLS) == declared_entry_points()


@pytest.mark.parametrize("name", ["D2Q33", "D3Q95"])
def test_model_info_matches_oracle(lbm, name):
    info = lbm.lbm_model_info(name)
    mdl = get_model(name)
    assert info["Q"] == mdl.Q and info["D"] == mdl.D and info["reach"] == mdl.reach
    assert abs(info["c"] - mdl.c) < 1e-14
    assert abs(info["T0"] - mdl.T0) < 1e-13
    # same set of velocities, weights per velocity agree
    ours = {tuple(v): w for v, w in zip(info["e"].tolist(), info["w"])}
    theirs = {tuple(v): w for v, w in zip(mdl.e.tolist(), mdl.w)}
    assert ours.keys() == theirs.keys()
    for k in ours:
        assert abs(ours[k] - theirs[k]) <= 1e-15 + 1e-13 * theirs[k]
    # storage order: rest first, then opposite pairs
    e = info["e"]
    assert not e[0].any()
    assert np.array_equal(e[1::2], -e[2::2])


def test_invalid_arguments_fail_without_a_gpu(lbm):
    lib = lbm._lib
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    assert lib.lbm_create(ctypes.byref(h), 7, dims, 1.0, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(h), 1, dims, 2.0, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_create(ctypes.byref(h), 1, dims, 1.0, 9, None) == lbm.LBM_EINVAL
    bad = (ctypes.c_int64 * 3)(8, 8, 0)
    assert lib.lbm_create(ctypes.byref(h), 1, bad, 1.0, 1, None) == lbm.LBM_EINVAL
    d2 = (ctypes.c_int64 * 3)(8, 8, 2)
    assert lib.lbm_create(ctypes.byref(h), 0, d2, 1.0, 1, None) == lbm.LBM_EINVAL
    assert "D2Q33" in lbm.lbm_last_error()
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lbm.lbm_strerror(lbm.LBM_ESTATE) == "call out of order"
    assert lib.lbm_model_info(5, None, None, None, None, None, None, None) == lbm.LBM_EINVAL


def test_no_product_module_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1303_4624_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".inl")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), fn
                assert "oracle/" not in src, fn
