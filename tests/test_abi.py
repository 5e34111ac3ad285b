"""The C-ABI library loads and exports every entry point include/knor.h
declares; argument validation that needs no GPU behaves as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1606_08905_gb300 import build as kbuild
from paper_1606_08905_gb300 import knor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knor_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return knor.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("knor.h")
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert re.fullmatch(r"\d+\.\d+\.\d+", knor.version())


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    pts = np.zeros((4, 2), np.float32)
    for n, d, k in [(4, 2, 5), (0, 2, 1), (4, 0, 1), (4, 2, 0)]:
        st = lib.knor_create(pts.ctypes.data, n, d, k, 0, 1, None, ctypes.byref(out))
        assert st == knor.KNOR_ERR_ARG
        assert out.value is None
        assert lib.knor_last_error(None)
    st = lib.knor_create(None, 4, 2, 1, 0, 1, None, ctypes.byref(out))
    assert st == knor.KNOR_ERR_ARG


def test_null_context_calls_are_rejected(lib):
    assert lib.knor_iterate(None, None) == knor.KNOR_ERR_ARG
    assert lib.knor_reset(None) == knor.KNOR_ERR_ARG
    lib.knor_destroy(None)  # no-op


def test_batch_create_rejects_bad_instances_without_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    pts = np.zeros((4, 8), np.float32)
    ptrs = (ctypes.c_void_p * 1)(pts.ctypes.data)
    for n, d, k in [(4, 8, 5), (4, 12, 2), (4, 8, 0), (0, 8, 1), (400, 8, 257)]:
        st = lib.knor_batch_create(1, ptrs, (ctypes.c_int64 * 1)(n), (ctypes.c_int32 * 1)(d),
                                   (ctypes.c_int32 * 1)(k), 1, None, ctypes.byref(out))
        assert st == knor.KNOR_ERR_ARG
        assert out.value is None
        assert lib.knor_last_error(None)
    assert lib.knor_batch_create(0, ptrs, None, None, None, 1, None, ctypes.byref(out)) == knor.KNOR_ERR_ARG
    assert lib.knor_batch_iterate(None, None) == knor.KNOR_ERR_ARG
    lib.knor_batch_destroy(None)  # no-op


def test_create_rejects_an_unknown_init_without_touching_the_gpu(lib):
    X = np.zeros((10, 4), np.float32)
    out = ctypes.c_void_p()
    for bad in (3, -1):
        st = lib.knor_create(X.ctypes.data, 10, 4, 2, bad, 1, None, ctypes.byref(out))
        assert st == knor.KNOR_ERR_ARG and "init" in lib.knor_last_error(None).decode()
