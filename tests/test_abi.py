"""The C-ABI library loads and exports every entry point include/shape.h
declares; argument checks that need no GPU return the documented status."""
import ctypes
import os
import re

import pytest

import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import _binding as B
from paper_2607_20766_b300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build_shape()
    return shp.load_library()


def header_functions():
    with open(os.path.join(ROOT, "include", "shape.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert "overlap_estimate" in names and "tanimoto_screen" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def test_version_and_error_string(lib):
    assert lib.shp_version() == 6
    assert isinstance(lib.shp_last_error(), bytes)


def test_null_and_bad_arguments_rejected(lib):
    mc = B.ShpMC(1, 0, 1024, B.SYMMETRIC)
    assert lib.overlap_estimate(None, None, None, None, 1, None, ctypes.byref(mc), None, None, None) == -1
    assert b"NULL set" in lib.shp_last_error()
    assert lib.union_volume_estimate(None, None, 1, ctypes.byref(mc), None, None, None, None, None) == -1
    assert lib.fo_overlap(None, None, None, None, 1, None, None, None) == -1
    assert lib.tanimoto_screen(None, None, None, None, None, None, None, None, None, None, None) == -1
    assert lib.shp_screen_variants() >= 1
    out = ctypes.c_void_p()
    off = (ctypes.c_int32 * 2)(0, 1)
    assert lib.shape_set_load(None, None, None, 0.0, None, 1, None, ctypes.byref(out)) == -1
    assert lib.shape_set_load(None, None, None, 0.0, off, -1, None, ctypes.byref(out)) == -1
    bad = (ctypes.c_int32 * 2)(0, 65)
    assert lib.shape_set_load(None, None, None, 0.0, bad, 1, None, ctypes.byref(out)) == -4
    zero = (ctypes.c_int32 * 2)(0, 0)
    assert lib.shape_set_load(None, None, None, 0.0, zero, 1, None, ctypes.byref(out)) == -4
    assert lib.shape_set_free(None) == 0
    assert lib.shape_set_free_async(None, None) == 0
    assert lib.shape_set_info(None, None, None, None) == -1
    assert lib.shp_fail_next_allocations(-1) == -1
    assert lib.shp_fail_next_allocations(0) == 0
    assert lib.union_self_estimate(None, None, 1, ctypes.byref(mc), None, 0.0, 256, 1, None, None, None, None, None,
                                   None) == -1
    assert lib.fo_tanimoto_screen(None, None, None, None, None, None) == -1
    assert lib.prefilter_db_ids(None, None, 0, None, None) == -1
    n_ev = ctypes.c_int64()
    assert lib.shp_eval_probe(None, 0, None, 0, -1, 0, 8, None, ctypes.byref(n_ev), None) == -1
    assert lib.align_rigid(None, 0, None, None, 1, None, None, None, None, None, None, None, None) in (-1, -4)
