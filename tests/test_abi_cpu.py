"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/hps.h declares; host-side argument
validation rejects bad input before any device work."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2211_14969_b300 import build as B
from paper_2211_14969_b300 import hps

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hps.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hps.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hps_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("hps_build_leaves", "hps_condense", "hps_merge", "hps_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_version(lib):
    assert lib.hps_version() == 105


def _build(lib, p, boxes, kappa=1.0, out=True):
    p = np.ascontiguousarray(np.asarray(p, dtype=np.int32))
    boxes = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 4))
    desc = hps._LeafDesc(len(p), p.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), kappa)
    h = ctypes.c_void_p()
    st = lib.hps_build_leaves(ctypes.byref(desc), ctypes.byref(h) if out else None, None)
    return st, h


@pytest.mark.parametrize("p,box,kappa", [
    ([3], [0, 0, 1, 1], 1.0),          # p below HPS_PMIN
    ([43], [0, 0, 1, 1], 1.0),         # p above HPS_PMAX
    ([10], [0, 0, -1, 1], 1.0),        # negative width
    ([10], [0, 0, 1, 0], 1.0),         # zero height
    ([10], [0, float("nan"), 1, 1], 1.0),
    ([10], [0, 0, 1, 1], float("inf")),
])
def test_build_rejects_bad_description(lib, p, box, kappa):
    st, h = _build(lib, p, box, kappa)
    assert st == hps.HPS_ERR_ARG
    assert not h.value
    assert b"hps_build_leaves" in lib.hps_last_error(None)


def test_build_rejects_null_out_and_empty(lib):
    st, _ = _build(lib, [10], [0, 0, 1, 1], out=False)
    assert st == hps.HPS_ERR_ARG
    desc = hps._LeafDesc(0, None, None, 1.0)
    h = ctypes.c_void_p()
    assert lib.hps_build_leaves(ctypes.byref(desc), ctypes.byref(h), None) == hps.HPS_ERR_ARG


def test_null_plan_calls_are_argument_errors(lib):
    vp = ctypes.c_void_p
    assert lib.hps_condense(None, 0, vp(1), None, 0, 0.0, 0, None, vp(1), None, None, vp(1), None) == hps.HPS_ERR_ARG
    assert lib.hps_merge(None, 1, 1, vp(1), None, 0, None) == hps.HPS_ERR_ARG
    assert lib.hps_solve(None, vp(1), vp(1), None, 1, vp(1), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_nodes(None, vp(1), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_resolve(None, 0, vp(1), None, 1, vp(1), 0.0, 0, vp(1), vp(1), None) == hps.HPS_ERR_ARG
    assert lib.hps_leaf_recover(None, vp(1), None, 1, vp(1), vp(1), None) == hps.HPS_ERR_ARG
    assert lib.hps_condense_host(None, 0, vp(1), None, 0, 0.0, 0, None, vp(1), None, None, vp(1), 0,
                                 None) == hps.HPS_ERR_ARG
    assert lib.hps_set_merge_split(None, -1) == hps.HPS_ERR_ARG
    assert lib.hps_set_timing(None, 1) == hps.HPS_ERR_ARG
    assert lib.hps_last_launch_count(None) == 0
    lib.hps_destroy(None)   # no-op


def test_layout_offsets():
    lay = hps.Layout([4, 10, 20])
    assert list(lay.ni) == [4, 64, 324]
    assert list(lay.nb) == [8, 32, 72]
    assert lay.o_sb[-1] == 4 * 8 + 64 * 32 + 324 * 72
    assert lay.o_bb[2] == 64 + 32 * 32
    assert lay.o_p2[-1] == 16 + 100 + 400
