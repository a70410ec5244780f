"""The C-ABI library builds, loads without a GPU and exports every function
include/blockmgard.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "blockmgard.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_00205_gb300 import _build

    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for n in ["bm_compress", "bm_decompress", "bm_compress_bound", "bm_stream_info", "bm_error_string",
              "bm_decompose", "bm_recompose", "bm_huffman_encode", "bm_huffman_decode"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.bm_error_string.restype = ctypes.c_char_p
    assert lib.bm_error_string(4) == b"corrupt stream"
    lib.bm_compress_bound.restype = ctypes.c_size_t
    lib.bm_compress_bound.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    shp = (ctypes.c_int64 * 3)(65, 65, 65)
    assert lib.bm_compress_bound(3, shp, 0) == 256 + 4 * 65 ** 3
    assert lib.bm_compress_bound(3, shp, 1) == 256 + 8 * 65 ** 3
    # 1-D / 2-D fields and extents of 1 (neither blocked nor coarsened)
    unit = (ctypes.c_int64 * 3)(65, 1, 65)
    assert lib.bm_compress_bound(3, unit, 0) == 256 + 4 * 65 * 65
    assert lib.bm_compress_bound(2, shp, 0) == 256 + 4 * 65 * 65
    assert lib.bm_compress_bound(1, shp, 1) == 256 + 8 * 65
    # invalid: an extent of 0, more than 3 dimensions, a single value
    assert lib.bm_compress_bound(3, (ctypes.c_int64 * 3)(65, 0, 65), 0) == 0
    assert lib.bm_compress_bound(4, shp, 0) == 0
    assert lib.bm_compress_bound(3, (ctypes.c_int64 * 3)(1, 1, 1), 0) == 0


def test_stream_info_on_host_header(lib):
    """bm_stream_info parses an oracle-written header from host memory."""
    import numpy as np

    import fields
    import oracle

    u = fields.gaussian_bumps((12, 11, 10), seed=3)
    s = oracle.compress(u, 1e-2, rel=True, B=9, K=2, M=1)
    nd = ctypes.c_int(0)
    shp = (ctypes.c_int64 * 3)()
    dt = ctypes.c_int(-1)
    nc = ctypes.c_size_t(0)
    lib.bm_stream_info.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_size_t)]
    st = lib.bm_stream_info(s.ctypes.data, s.size, 0, ctypes.byref(nd), shp, ctypes.byref(dt), ctypes.byref(nc))
    assert st == 0
    assert tuple(shp) == (12, 11, 10) and dt.value == 0 and nd.value == 3
    assert nc.value == oracle.plan((12, 11, 10), 9, 2, 1)["n_coeffs"]
    t = s.copy()
    t[0] ^= 0xFF
    assert lib.bm_stream_info(t.ctypes.data, t.size, 0, None, None, None, None) == 4
    assert lib.bm_stream_info(s.ctypes.data, s.size - 8, 0, None, None, None, None) == 4
    del np


def test_stream_info_on_2d_header(lib):
    """A 2-D field's stream: bm_stream_info reports 2 dimensions and the
    field's own extents first."""
    import numpy as np

    import oracle

    u = np.random.default_rng(1).normal(size=(40, 23)).astype(np.float32)
    s = oracle.compress(u, 1e-2, rel=True, B=9, K=2, M=1)
    nd = ctypes.c_int(0)
    shp = (ctypes.c_int64 * 3)()
    dt = ctypes.c_int(-1)
    nc = ctypes.c_size_t(0)
    lib.bm_stream_info.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_size_t)]
    assert lib.bm_stream_info(s.ctypes.data, s.size, 0, ctypes.byref(nd), shp, ctypes.byref(dt), ctypes.byref(nc)) == 0
    assert nd.value == 2 and list(shp) == [40, 23, 0] and dt.value == 0
    assert nc.value == oracle.plan((40, 23), 9, 2, 1)["n_coeffs"]
