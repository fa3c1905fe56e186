"""The C-ABI library builds, loads and exports every entry point of include/lk.h.

These run without a GPU: only calls that fail on argument checks before any
device work are made.
"""
import os
import re

import numpy as np
import pytest

from paper_2106_12655_gb300 import build as B
from paper_2106_12655_gb300 import lk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "lk.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lk_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lk.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lk_create", "lk_verify", "lk_update", "lk_destroy", "lk_sync", "lk_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if not hasattr(lk, n)]
    assert not missing, missing


def test_default_options(lib):
    o = lk.lk_default_options()
    assert o.precision == lk.LK_MIXED
    assert o.near_ratio == 3.0
    assert o.int_tol == 0.1
    assert o.near_capacity == 1 << 20
    assert o.method == lk.LK_METHOD_DS and o.cc_capacity == 1 << 18
    assert o.cc_search == lk.LK_CC_SEARCH_AUTO


def _create_status(v, off, opt=None):
    with pytest.raises(lk.LkError) as ei:
        lk.lk_create(v, off, opt)
    return ei.value.status


def test_create_rejects_bad_geometry_before_device_work(lib):
    v = np.random.default_rng(0).normal(size=(10, 3))
    assert _create_status(v, np.array([0, 2, 10], np.int64)) == lk.LK_ERR_ARG       # loop of 2
    assert _create_status(v, np.array([0, 5, 9], np.int64)) == lk.LK_ERR_ARG        # does not end at N
    assert _create_status(v, np.array([1, 5, 10], np.int64)) == lk.LK_ERR_ARG       # does not start at 0
    bad = v.copy()
    bad[3, 1] = np.nan
    assert _create_status(bad, np.array([0, 5, 10], np.int64)) == lk.LK_ERR_ARG
    o = lk.lk_default_options()
    o.near_ratio = 2.5
    assert _create_status(v, np.array([0, 5, 10], np.int64), o) == lk.LK_ERR_ARG
    o = lk.lk_default_options()
    o.method = lk.LK_METHOD_CC
    o.precision = lk.LK_ALL_F64                       # counting crossings needs LK_MIXED
    assert _create_status(v, np.array([0, 5, 10], np.int64), o) == lk.LK_ERR_ARG
    o = lk.lk_default_options()
    o.method = 7
    assert _create_status(v, np.array([0, 5, 10], np.int64), o) == lk.LK_ERR_ARG
    for bad_search in (-1, 3):
        o = lk.lk_default_options()
        o.method = lk.LK_METHOD_CC
        o.cc_search = bad_search
        assert _create_status(v, np.array([0, 5, 10], np.int64), o) == lk.LK_ERR_ARG


def test_create_rejects_zero_length_segments(lib):
    v = np.random.default_rng(1).normal(size=(10, 3))
    v[7] = v[6]
    assert _create_status(v, np.array([0, 5, 10], np.int64)) == lk.LK_ERR_ZERO_SEGMENT
    v = np.random.default_rng(1).normal(size=(10, 3)).astype(np.float32)
    v[9] = v[5]                          # closing segment of loop 1 (vertex 9 -> vertex 5)
    assert _create_status(v, np.array([0, 5, 10], np.int64)) == lk.LK_ERR_ZERO_SEGMENT
    assert "zero-length" in lk.lk_last_error()


def test_null_context_calls_fail_cleanly(lib):
    pairs = np.zeros((1, 2), np.int32)
    with pytest.raises(lk.LkError) as ei:
        lk.lk_verify(None, pairs)
    assert ei.value.status == lk.LK_ERR_ARG
    lk.lk_destroy(None)
    lk.lk_plan_destroy(None)
