"""CPU oracle for the BlockMGARD hot path — TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``liboracle.so`` (built from ``oracle.cpp`` by
:func:`build`).  Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline / reference leg may import this package; the CUDA library and its
Python binding never do.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

HEADER_BYTES = 256


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FP contraction, so results are the same
    on x86-64 and aarch64 hosts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # OR_LIBRARY: a build of a modified oracle source (the planted-mistake
        # tests run the pins against such builds); otherwise the in-tree build
        path = os.environ.get("OR_LIBRARY")
        if not path:
            path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i64, u8 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint8
        L.or_last_error.restype = ctypes.c_char_p
        L.or_level_1d.argtypes = [ctypes.c_int, P(d), P(d), P(d), P(d), P(d), P(ctypes.c_int)]
        L.or_plan.argtypes = [P(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(i64)]
        L.or_decompose.argtypes = [P(d), P(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d)]
        L.or_recompose.argtypes = [P(d), P(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d)]
        L.or_block_coeffs.argtypes = [P(d), P(i64), ctypes.c_int, ctypes.c_int, i64, P(d), P(d)]
        L.or_level_constants.argtypes = [P(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d)]
        L.or_budget.argtypes = [P(i64), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d), ctypes.c_int, d,
                                ctypes.c_int, P(d), P(d)]
        L.or_quantize.argtypes = [d, d, ctypes.c_int, P(ctypes.c_int)]
        L.or_quantize.restype = i64
        L.or_quantize_array.argtypes = [P(d), P(d), i64, ctypes.c_int, P(i64), P(u8)]
        L.or_huffman_lengths.argtypes = [P(ctypes.c_uint64), ctypes.c_int, P(u8)]
        L.or_canonical_codes.argtypes = [P(u8), ctypes.c_int, P(ctypes.c_uint32)]
        L.or_huffman_encode.argtypes = [P(ctypes.c_uint16), ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P(u8),
                                        ctypes.c_uint64, P(ctypes.c_uint64)]
        L.or_huffman_decode.argtypes = [P(u8), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, P(ctypes.c_uint32),
                                        P(ctypes.c_uint32), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        P(ctypes.c_uint16)]
        L.or_compress.argtypes = [P(d), P(i64), ctypes.c_int, d, ctypes.c_int, P(d), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, P(u8), ctypes.c_uint64,
                                  P(ctypes.c_uint64), P(i64)]
        L.or_decompress.argtypes = [P(u8), ctypes.c_uint64, P(d), P(i64)]
        ci = ctypes.c_int
        L.or_plan_r.argtypes = [P(i64), ci, ci, ci, ci, P(i64)]
        L.or_decompose_r.argtypes = [P(d), P(i64), ci, ci, ci, ci, P(d)]
        L.or_recompose_r.argtypes = [P(d), P(i64), ci, ci, ci, ci, P(d)]
        L.or_rounds.argtypes = [P(i64), ci, ci, ci, P(u8), P(i64), P(u8)]
        L.or_budget_r.argtypes = [P(i64), ci, ci, ci, ci, P(d), ci, d, ci, P(d), P(d)]
        L.or_compress_r.argtypes = [P(d), P(i64), ci, d, ci, P(d), ci, ci, ci, ci, ci, ci, P(u8), ctypes.c_uint64,
                                    P(ctypes.c_uint64), P(i64)]
        L.or_compress_nd.argtypes = [P(d), P(i64), ci, ci, d, ci, P(d), ci, ci, ci, ci, ci, ci, P(u8),
                                     ctypes.c_uint64, P(ctypes.c_uint64), P(i64)]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle: " + lib().or_last_error().decode())


def _shape3(shape):
    """A shape of 1..3 dimensions as a 3-D shape with leading extents of 1 (the
    missing dimensions are neither blocked nor coarsened)."""
    s = [int(v) for v in shape]
    if not 1 <= len(s) <= 3:
        raise ValueError("fields have 1, 2 or 3 dimensions")
    return np.ascontiguousarray(np.array([1] * (3 - len(s)) + s, dtype=np.int64))


# ---------------------------------------------------------------------------
def level_1d(x):
    """1-D operators for node coordinates x: (I, Mf, Mc, P) as dense arrays."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n = x.size
    nc = n // 2 + 1
    I = np.zeros((n, nc)); Mf = np.zeros((n, n)); Mc = np.zeros((nc, nc)); P = np.zeros((nc, n))
    out_nc = ctypes.c_int(0)
    c = ctypes.c_double
    _check(lib().or_level_1d(n, _ptr(x, c), _ptr(I, c), _ptr(Mf, c), _ptr(Mc, c), _ptr(P, c), ctypes.byref(out_nc)))
    assert out_nc.value == nc
    return I, Mf, Mc, P


def plan(shape, B, K, M, R=1):
    out = np.zeros(11 + max(M, 1), dtype=np.int64)
    _check(lib().or_plan_r(_ptr(_shape3(shape), ctypes.c_int64), B, K, M, R, _ptr(out, ctypes.c_int64)))
    return {
        "n_coeffs": int(out[0]), "per_block": int(out[1]), "nblocks": int(out[2]), "m": int(out[3]),
        "gshape": tuple(int(v) for v in out[4:7]), "cshape": tuple(int(v) for v in out[7:10]),
        "coarsest": int(out[10]), "global_counts": [int(v) for v in out[11:11 + M]],
    }


def decompose(u, B, K, M, R=1):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    p = plan(u.shape, B, K, M, R)
    coef = np.zeros(p["n_coeffs"])
    c = ctypes.c_double
    _check(lib().or_decompose_r(_ptr(u, c), _ptr(_shape3(u.shape), ctypes.c_int64), B, K, M, R, _ptr(coef, c)))
    return coef


def recompose(coef, shape, B, K, M, R=1):
    coef = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    u = np.zeros(tuple(shape))
    c = ctypes.c_double
    _check(lib().or_recompose_r(_ptr(coef, c), _ptr(_shape3(shape), ctypes.c_int64), B, K, M, R, _ptr(u, c)))
    return u


def rounds(shape, B, K, R, tier0=None):
    """Blocks of every re-blocking round and, given round 0's block tiers,
    every round's propagated tiers (a list of arrays)."""
    nb = np.zeros(R, dtype=np.int64)
    t0 = None if tier0 is None else np.ascontiguousarray(np.asarray(tier0, dtype=np.uint8))
    out = None
    if t0 is not None:
        out = np.zeros(int(sum(plan_rounds_count(shape, B, K, R))), dtype=np.uint8)
    _check(lib().or_rounds(_ptr(_shape3(shape), ctypes.c_int64), B, K, R,
                           _ptr(t0, ctypes.c_uint8) if t0 is not None else None, _ptr(nb, ctypes.c_int64),
                           _ptr(out, ctypes.c_uint8) if out is not None else None))
    if out is None:
        return [int(v) for v in nb], None
    parts, o = [], 0
    for v in nb:
        parts.append(out[o:o + int(v)])
        o += int(v)
    return [int(v) for v in nb], parts


def plan_rounds_count(shape, B, K, R):
    nb = np.zeros(R, dtype=np.int64)
    _check(lib().or_rounds(_ptr(_shape3(shape), ctypes.c_int64), B, K, R, None, _ptr(nb, ctypes.c_int64), None))
    return [int(v) for v in nb]


def decompose_matrix(shape, B, K, M):
    """The decomposition as an explicit matrix (n_coeffs x prod(shape)), built
    column by column from unit inputs: the plain definition of the operator
    whose transpose the adjoint kernels must equal (small grids only)."""
    shape = tuple(int(v) for v in shape)
    n = int(np.prod(shape))
    A = np.zeros((plan(shape, B, K, M)["n_coeffs"], n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = decompose(e.reshape(shape), B, K, M)
        e[j] = 0.0
    return A


def recompose_matrix(shape, B, K, M):
    """The recomposition as an explicit matrix (prod(shape) x n_coeffs)."""
    shape = tuple(int(v) for v in shape)
    nc = plan(shape, B, K, M)["n_coeffs"]
    R = np.zeros((int(np.prod(shape)), nc))
    e = np.zeros(nc)
    for j in range(nc):
        e[j] = 1.0
        R[:, j] = recompose(e, shape, B, K, M).ravel()
        e[j] = 0.0
    return R


def decompose_adjoint(coef_grad, shape, B, K, M):
    """Transpose of the decomposition applied to coefficient gradients."""
    return (decompose_matrix(shape, B, K, M).T @ np.asarray(coef_grad, dtype=np.float64)).reshape(shape)


def recompose_adjoint(field_grad, shape, B, K, M):
    """Transpose of the recomposition applied to field gradients."""
    return recompose_matrix(shape, B, K, M).T @ np.asarray(field_grad, dtype=np.float64).ravel()


def block_coeffs(u, B, K, block):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    p = plan(u.shape, B, K, 0)
    coef = np.zeros(p["per_block"])
    coarse = np.zeros(p["m"] ** 3)
    c = ctypes.c_double
    _check(lib().or_block_coeffs(_ptr(u, c), _ptr(_shape3(u.shape), ctypes.c_int64), B, K, int(block),
                                 _ptr(coef, c), _ptr(coarse, c)))
    return coef, coarse.reshape((p["m"],) * 3)


def level_constants(shape, B, K, M):
    out = np.zeros(K + M)
    _check(lib().or_level_constants(_ptr(_shape3(shape), ctypes.c_int64), B, K, M, _ptr(out, ctypes.c_double)))
    return out


def budget(shape, B, K, M, taus, max_abs, f64, R=1):
    taus = np.ascontiguousarray(np.asarray(taus, dtype=np.float64))
    q = np.zeros(len(taus) * K + M + 1)
    meta = np.zeros(2)
    c = ctypes.c_double
    _check(lib().or_budget_r(_ptr(_shape3(shape), ctypes.c_int64), B, K, M, R, _ptr(taus, c), len(taus),
                             float(max_abs), int(bool(f64)), _ptr(q, c), _ptr(meta, c)))
    return q, float(meta[0]), bool(meta[1])


def quantize(c, q, f64):
    ov = ctypes.c_int(0)
    code = lib().or_quantize(float(c), float(q), int(bool(f64)), ctypes.byref(ov))
    return int(code), bool(ov.value)


def quantize_array(c, q, f64):
    """The quantiser over arrays of coefficients and bin widths: (codes,
    overflow flags)."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    q = np.ascontiguousarray(np.broadcast_to(np.asarray(q, dtype=np.float64), c.shape))
    codes = np.zeros(c.size, dtype=np.int64)
    ovf = np.zeros(c.size, dtype=np.uint8)
    _check(lib().or_quantize_array(_ptr(c, ctypes.c_double), _ptr(q, ctypes.c_double), c.size, int(bool(f64)),
                                   _ptr(codes, ctypes.c_int64), _ptr(ovf, ctypes.c_uint8)))
    return codes.reshape(c.shape), ovf.astype(bool).reshape(c.shape)


def huffman_lengths(freq):
    f = np.ascontiguousarray(np.asarray(freq, dtype=np.uint64))
    out = np.zeros(f.size, dtype=np.uint8)
    _check(lib().or_huffman_lengths(_ptr(f, ctypes.c_uint64), f.size, _ptr(out, ctypes.c_uint8)))
    return out


def canonical_codes(lengths):
    l = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    out = np.zeros(l.size, dtype=np.uint32)
    _check(lib().or_canonical_codes(_ptr(l, ctypes.c_uint8), l.size, _ptr(out, ctypes.c_uint32)))
    return out


def huffman_encode(sym, dict_size, chunk):
    """Huffman section bytes (chunk word counts | split offsets | codebook
    runs | words) and its sizes dict."""
    s = np.ascontiguousarray(np.asarray(sym, dtype=np.uint16))
    cap = 64 + 8 * s.size + 8 * dict_size + 24 * (s.size // max(chunk, 1) + 2)
    out = np.zeros(cap, dtype=np.uint8)
    sizes = np.zeros(5, dtype=np.uint64)
    _check(lib().or_huffman_encode(_ptr(s, ctypes.c_uint16), s.size, dict_size, chunk, _ptr(out, ctypes.c_uint8),
                                   cap, _ptr(sizes, ctypes.c_uint64)))
    meta = {"codebook_bytes": int(sizes[0]), "n_runs": int(sizes[1]), "n_chunks": int(sizes[2]),
            "n_words": int(sizes[3]), "bytes": int(sizes[4])}
    return out[:meta["bytes"]].copy(), meta


def huffman_decode(section, meta, n, dict_size, chunk):
    sec = np.ascontiguousarray(np.asarray(section, dtype=np.uint8))
    cb = meta["codebook_bytes"]
    off_cb = (4 * meta["n_chunks"] + 7) // 8 * 8 + (14 * meta["n_chunks"] + 7) // 8 * 8
    off_w = off_cb + (cb + 7) // 8 * 8
    chunks = np.ascontiguousarray(sec[:4 * meta["n_chunks"]].view(np.uint32))
    words = np.ascontiguousarray(sec[off_w:off_w + 4 * meta["n_words"]].view(np.uint32))
    cbk = np.ascontiguousarray(sec[off_cb:off_cb + cb])
    out = np.zeros(n, dtype=np.uint16)
    _check(lib().or_huffman_decode(_ptr(cbk, ctypes.c_uint8), cb, meta["n_runs"], dict_size,
                                   _ptr(chunks, ctypes.c_uint32), _ptr(words, ctypes.c_uint32), meta["n_words"], n,
                                   chunk, _ptr(out, ctypes.c_uint16)))
    return out


def compress(u, tol, rel=True, roi=None, B=9, K=1, M=2, chunk=2048, radius=32768, f64=None, want_codes=False, R=1):
    """Full stream for field u (numpy, float32 or float64).  Returns bytes
    (uint8 array) and, if asked, the integer codes in coefficient order."""
    if f64 is None:
        f64 = np.asarray(u).dtype == np.float64
    u64 = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    p = plan(u64.shape, B, K, M, R)
    cap = HEADER_BYTES + 8 * u64.size + 16 * p["n_coeffs"] + 2 * sum(plan_rounds_count(u64.shape, B, K, R)) \
        + 16 * radius + (1 << 16)
    out = np.zeros(cap, dtype=np.uint8)
    nbytes = ctypes.c_uint64(0)
    roi_arr = None
    if roi is not None:
        roi_arr = np.ascontiguousarray(np.asarray(roi, dtype=np.float64).ravel())
        assert roi_arr.size == p["nblocks"]
    codes = np.zeros(p["n_coeffs"], dtype=np.int64) if want_codes else None
    c = ctypes.c_double
    rc = lib().or_compress_nd(_ptr(u64, c), _ptr(_shape3(u64.shape), ctypes.c_int64), u64.ndim, int(bool(f64)),
                              float(tol), int(bool(rel)), _ptr(roi_arr, c) if roi_arr is not None else None, B, K, M,
                              R, chunk, radius, _ptr(out, ctypes.c_uint8), cap, ctypes.byref(nbytes),
                              _ptr(codes, ctypes.c_int64) if codes is not None else None)
    _check(rc)
    s = out[:nbytes.value].copy()
    return (s, codes) if want_codes else s


def decompress(stream, want_codes=False):
    s = np.ascontiguousarray(np.asarray(stream, dtype=np.uint8))
    info = stream_header(s)
    u = np.zeros(info["shape"])  # the 3-D shape; reshaped to the field's own dimensions below
    codes = None
    if want_codes and not info["raw"]:
        codes = np.zeros(int(info["n_symbols"]), dtype=np.int64)
    _check(lib().or_decompress(_ptr(s, ctypes.c_uint8), s.size, _ptr(u, ctypes.c_double),
                               _ptr(codes, ctypes.c_int64) if codes is not None else None))
    u = u.astype(np.float64 if info["f64"] else np.float32)
    nd = info["ndim"] if 1 <= info["ndim"] <= 3 else 3
    u = u.reshape(info["shape"][3 - nd:])
    return (u, codes) if want_codes else u


def stream_header(s):
    """Parse the fixed 256-byte header (field names as in the stream format)."""
    s = np.asarray(s, dtype=np.uint8)
    h = s[:HEADER_BYTES].tobytes()
    import struct
    magic, version, flags = struct.unpack_from("<IHH", h, 0)
    if magic != 0x31474D42:
        raise ValueError("not a BlockMGARD stream")
    i32 = lambda o: struct.unpack_from("<i", h, o)[0]
    i64 = lambda o: struct.unpack_from("<q", h, o)[0]
    u64 = lambda o: struct.unpack_from("<Q", h, o)[0]
    u32 = lambda o: struct.unpack_from("<I", h, o)[0]
    f64 = lambda o: struct.unpack_from("<d", h, o)[0]
    return {
        "version": version, "flags": flags, "raw": bool(flags & 1), "f64": bool(flags & 2),
        "ndim": i32(8), "B": i32(12), "shape": (i64(16), i64(24), i64(32)), "K": i32(40), "M": i32(44),
        "chunk": i32(48), "radius": i32(52), "n_tiers": i32(56), "m": i32(60),
        "nb": (i32(64), i32(68), i32(72)), "rel": i32(76), "max_abs": f64(80), "tol": f64(88),
        "n_symbols": u64(96), "n_chunks": u64(104), "n_outliers": u64(112), "n_words": u64(120),
        "off_tiers": u64(128), "off_qtab": u64(136), "off_blocktier": u64(144), "off_chunks": u64(152),
        "off_codebook": u64(160), "off_bits": u64(168), "off_outliers": u64(176), "total": u64(184),
        "codebook_bytes": u32(192), "n_runs": u32(196), "margin": f64(200), "off_chunk_esc": u64(208),
        "off_splits": u64(216), "R": u32(224) + 1,
    }
