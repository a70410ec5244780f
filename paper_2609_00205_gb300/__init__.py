"""BlockMGARD on GB300: Python binding of the C-ABI library ``libbm.so``.

Only argument marshalling lives here: every step of compression and
decompression runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library is missing or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

__all__ = [
    "BM_F32", "BM_F64", "BlockMGARDError", "load", "compress", "compress_batch", "decompress", "decompose", "recompose",
    "coeff_count", "stream_info", "stream_codes", "huffman_encode", "huffman_decode", "compress_bound",
    "set_timing", "stage_times", "stage_timeline", "decompose_adjoint", "recompose_adjoint", "Decompose",
    "Recompose", "decompose_ad", "recompose_ad", "PerfModel", "perf_model_fit", "perf_model_knee", "predict_ms",
    "select_params", "launch_count", "release_workspace", "library_path",
]

BM_F32, BM_F64 = 0, 1
BM_ABS, BM_REL = 0, 1
_STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "output capacity too small", 4: "corrupt stream",
           5: "unsupported", 6: "out of device memory"}


class BlockMGARDError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__("%s: %s" % (_STATUS.get(status, "status %d" % status), detail))
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("block_nodes", ctypes.c_int), ("incache_levels", ctypes.c_int), ("global_levels", ctypes.c_int),
                ("chunk_symbols", ctypes.c_int), ("dict_radius", ctypes.c_int), ("rounds", ctypes.c_int)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("d_field", ctypes.c_void_p), ("ndim", ctypes.c_int), ("shape", ctypes.c_int64 * 3),
                ("dtype", ctypes.c_int), ("tol", ctypes.c_double), ("tol_mode", ctypes.c_int),
                ("h_roi_tol", ctypes.POINTER(ctypes.c_double)), ("params", _Params), ("d_out", ctypes.c_void_p),
                ("out_capacity", ctypes.c_size_t)]


class PerfModel(ctypes.Structure):
    """Fitted performance model (Eq. 1 for the In-cache Block stage, lines for
    the rest); see bm_perf_model in include/blockmgard.h."""
    _fields_ = [("block_latency_ms", ctypes.c_double), ("block_peak_per_ms", ctypes.c_double),
                ("global_ms", ctypes.c_double), ("global_ms_per_node", ctypes.c_double),
                ("hist_ms", ctypes.c_double), ("hist_ms_per_symbol", ctypes.c_double),
                ("codebook_ms", ctypes.c_double), ("encode_ms", ctypes.c_double),
                ("encode_ms_per_symbol", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("block_nodes", ctypes.c_int), ("incache_levels", ctypes.c_int), ("dtype", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    """libbm.so in the package tree; BM_LIBRARY overrides it (a build of the
    same sources with other compile-time options)."""
    return os.environ.get("BM_LIBRARY", _build.LIB)


def load():
    """Load libbm.so (built by ``__graft_entry__.build()`` / ``_build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libbm.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, sz, i64, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_uint64
    L.bm_compress_bound.argtypes = [ctypes.c_int, P(i64), ctypes.c_int]
    L.bm_compress_bound.restype = sz
    L.bm_compress.argtypes = [vp, ctypes.c_int, P(i64), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                              P(ctypes.c_double), P(_Params), vp, sz, P(sz), vp]
    L.bm_stream_info.argtypes = [vp, sz, ctypes.c_int, P(ctypes.c_int), P(i64), P(ctypes.c_int), P(sz)]
    L.bm_decompress.argtypes = [vp, sz, vp, vp]
    L.bm_compress_batch.argtypes = [ctypes.c_int, P(_BatchItem), P(sz), P(ctypes.c_int), vp]
    L.bm_perf_model_fit.argtypes = [ctypes.c_int, ctypes.c_int, P(PerfModel), vp]
    L.bm_perf_model_knee.argtypes = [P(PerfModel), ctypes.c_double]
    L.bm_perf_model_knee.restype = ctypes.c_double
    L.bm_predict_ms.argtypes = [P(PerfModel), ctypes.c_int, P(i64), P(_Params), P(ctypes.c_double)]
    L.bm_select_params.argtypes = [P(PerfModel), ctypes.c_int, P(i64), ctypes.c_double, P(_Params),
                                   P(ctypes.c_double)]
    L.bm_decompose.argtypes = [vp, ctypes.c_int, P(i64), ctypes.c_int, P(_Params), vp, vp]
    L.bm_recompose.argtypes = [vp, ctypes.c_int, P(i64), ctypes.c_int, P(_Params), vp, vp]
    L.bm_decompose_adjoint.argtypes = [vp, ctypes.c_int, P(i64), ctypes.c_int, P(_Params), vp, vp]
    L.bm_recompose_adjoint.argtypes = [vp, ctypes.c_int, P(i64), ctypes.c_int, P(_Params), vp, vp]
    L.bm_coeff_count.argtypes = [ctypes.c_int, P(i64), P(_Params), P(sz)]
    L.bm_stream_codes.argtypes = [vp, sz, vp, vp]
    L.bm_huffman_encode.argtypes = [vp, u64, ctypes.c_int, ctypes.c_int, vp, sz, P(u64), vp]
    L.bm_huffman_decode.argtypes = [vp, P(u64), u64, ctypes.c_int, ctypes.c_int, vp, vp]
    L.bm_release_workspace.argtypes = [vp]
    L.bm_release_workspace.restype = None
    L.bm_set_timing.argtypes = [ctypes.c_int]
    L.bm_set_timing.restype = None
    L.bm_set_block_grid_limit.argtypes = [ctypes.c_int]
    L.bm_set_block_grid_limit.restype = None
    L.bm_stage_times.argtypes = [P(ctypes.c_char_p), P(ctypes.c_float), ctypes.c_int]
    L.bm_stage_timeline.argtypes = [P(ctypes.c_char_p), P(ctypes.c_float), P(ctypes.c_float), ctypes.c_int]
    L.bm_launch_count.restype = u64
    L.bm_error_string.restype = ctypes.c_char_p
    L.bm_last_error_detail.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise BlockMGARDError(status, load().bm_last_error_detail().decode())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _shape(shape):
    """Extents of a field of 1..3 dimensions (a C array of 3; unused entries 0)."""
    s = [int(v) for v in shape]
    if not 1 <= len(s) <= 3:
        raise ValueError("fields have 1, 2 or 3 dimensions")
    return (ctypes.c_int64 * 3)(*(s + [0] * (3 - len(s))))


def _dtype(t):
    if t == torch.float32:
        return BM_F32
    if t == torch.float64:
        return BM_F64
    raise TypeError("fields must be float32 or float64")


def _params(block=17, levels=2, global_levels=2, chunk=2048, radius=32768, rounds=1):
    return _Params(int(block), int(levels), int(global_levels) if global_levels != 0 else -1, int(chunk), int(radius),
                   int(rounds))


def _dev_check(t):
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")


def compress_bound(shape, dtype=torch.float32) -> int:
    return int(load().bm_compress_bound(len(shape), _shape(shape), _dtype(dtype)))


def compress(field: torch.Tensor, tol: float, mode: str = "rel", roi=None, block=17, levels=2, global_levels=2,
             chunk=2048, radius=32768, out: torch.Tensor | None = None, stream=None, rounds=1) -> torch.Tensor:
    """Compress a 3-D float32/float64 CUDA tensor; returns the stream as a
    uint8 CUDA tensor (a view of ``out`` when given).  ``roi``: optional
    per-block tolerances (same mode as ``tol``), row-major over the block grid."""
    _dev_check(field)
    if not 1 <= field.dim() <= 3:
        raise ValueError("fields have 1, 2 or 3 dimensions")
    L = load()
    cap = compress_bound(field.shape, field.dtype)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    elif out.numel() < cap or out.dtype != torch.uint8 or not out.is_cuda:
        raise ValueError("out must be a CUDA uint8 tensor of at least compress_bound() bytes")
    roi_ptr = None
    if roi is not None:
        import numpy as np
        r = np.ascontiguousarray(np.asarray(roi, dtype=np.float64).ravel())
        roi_ptr = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nbytes = ctypes.c_size_t(0)
    p = _params(block, levels, global_levels, chunk, radius, rounds)
    with torch.cuda.device(field.device):
        _check(L.bm_compress(ctypes.c_void_p(field.data_ptr()), field.dim(), _shape(field.shape), _dtype(field.dtype),
                             float(tol), BM_REL if mode == "rel" else BM_ABS, roi_ptr, ctypes.byref(p),
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_size_t(out.numel()), ctypes.byref(nbytes),
                             _stream(stream)))
    return out[: nbytes.value]


def compress_batch(fields, tols, mode: str = "rel", rois=None, block=17, levels=2, global_levels=2, chunk=2048,
                   radius=32768, outs=None, stream=None, rounds=1, params=None):
    """Compress several CUDA fields (1-3 dims) in one call: the In-cache Block
    stage of every 3-D field with B in {9, 17} and one round runs in one
    persistent launch per (dtype, B, K), the rest of each pipeline on the
    library's stream pool, one synchronisation.  ``tols``: one tolerance per
    field; ``rois``: None or one per-block tolerance map (or None) per field;
    ``outs``: optional output buffers; ``params``: None or one dict per field
    (keys block, levels, global_levels, chunk, radius, rounds) overriding the
    shared keyword arguments.  Returns the streams as uint8 views, each
    identical to :func:`compress` of the same field and parameters."""
    import numpy as np
    L = load()
    n = len(fields)
    if (len(tols) != n or (rois is not None and len(rois) != n) or (outs is not None and len(outs) != n)
            or (params is not None and len(params) != n)):
        raise ValueError("one tolerance (and ROI map, output, parameter set) per field")
    shared = dict(block=block, levels=levels, global_levels=global_levels, chunk=chunk, radius=radius, rounds=rounds)
    items = (_BatchItem * max(n, 1))()
    keep = []
    bufs = []
    p = _params(block, levels, global_levels, chunk, radius, rounds)
    for i, f in enumerate(fields):
        _dev_check(f)
        if not 1 <= f.dim() <= 3:
            raise ValueError("fields have 1, 2 or 3 dimensions")
        cap = compress_bound(f.shape, f.dtype)
        o = outs[i] if outs is not None else torch.empty(cap, dtype=torch.uint8, device=f.device)
        if o.numel() < cap or o.dtype != torch.uint8 or not o.is_cuda:
            raise ValueError("out must be a CUDA uint8 tensor of at least compress_bound() bytes")
        bufs.append(o)
        it = items[i]
        it.d_field = f.data_ptr()
        it.ndim = f.dim()
        for d in range(3):
            it.shape[d] = int(f.shape[d]) if d < f.dim() else 0
        it.dtype = _dtype(f.dtype)
        it.tol = float(tols[i])
        it.tol_mode = BM_REL if mode == "rel" else BM_ABS
        r = rois[i] if rois is not None else None
        if r is not None:
            r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).ravel())
            keep.append(r)
            it.h_roi_tol = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if params is not None and params[i]:
            q = dict(shared, **params[i])
            it.params = _params(q["block"], q["levels"], q["global_levels"], q["chunk"], q["radius"], q["rounds"])
        else:
            it.params = p
        it.d_out = o.data_ptr()
        it.out_capacity = o.numel()
    sizes = (ctypes.c_size_t * max(n, 1))()
    status = (ctypes.c_int * max(n, 1))()
    dev = fields[0].device if n else torch.device("cuda", torch.cuda.current_device())
    with torch.cuda.device(dev):
        _check(L.bm_compress_batch(n, items, sizes, status, _stream(stream)))
    return [bufs[i][: sizes[i]] for i in range(n)]


def perf_model_fit(dtype=torch.float32, block=17, stream=None) -> PerfModel:
    """Calibrate the performance model on the current GPU (synchronous)."""
    m = PerfModel()
    _check(load().bm_perf_model_fit(_dtype(dtype), int(block), ctypes.byref(m), _stream(stream)))
    return m


def perf_model_knee(model: PerfModel, fraction: float = 0.9) -> float:
    return float(load().bm_perf_model_knee(ctypes.byref(model), float(fraction)))


def predict_ms(model: PerfModel, shape, block=17, levels=2, global_levels=2) -> float:
    ms = ctypes.c_double(0.0)
    p = _params(block, levels, global_levels)
    _check(load().bm_predict_ms(ctypes.byref(model), 3, _shape(shape), ctypes.byref(p), ctypes.byref(ms)))
    return ms.value


def select_params(model: PerfModel, shape, budget_ms: float):
    """Alg. 1: (block, levels, global_levels) maximising (M, -K) within the
    time budget; returns (params dict, predicted ms)."""
    p = _Params()
    ms = ctypes.c_double(0.0)
    _check(load().bm_select_params(ctypes.byref(model), 3, _shape(shape), float(budget_ms), ctypes.byref(p),
                                   ctypes.byref(ms)))
    return {"block": p.block_nodes, "levels": p.incache_levels,
            "global_levels": p.global_levels if p.global_levels > 0 else 0}, ms.value


def stream_info(buf: torch.Tensor) -> dict:
    L = load()
    nd = ctypes.c_int(0)
    shp = (ctypes.c_int64 * 3)()
    dt = ctypes.c_int(0)
    nc = ctypes.c_size_t(0)
    if buf.is_cuda:
        with torch.cuda.device(buf.device):
            _check(L.bm_stream_info(ctypes.c_void_p(buf.data_ptr()), buf.numel(), 1, ctypes.byref(nd), shp,
                                    ctypes.byref(dt), ctypes.byref(nc)))
    else:
        b = buf.contiguous()
        _check(L.bm_stream_info(ctypes.c_void_p(b.data_ptr()), b.numel(), 0, ctypes.byref(nd), shp, ctypes.byref(dt),
                                ctypes.byref(nc)))
    return {"shape": tuple(shp[: nd.value]), "dtype": torch.float64 if dt.value == BM_F64 else torch.float32,
            "n_coeffs": nc.value}


def decompress(buf: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _dev_check(buf)
    L = load()
    info = stream_info(buf)
    if out is None:
        out = torch.empty(info["shape"], dtype=info["dtype"], device=buf.device)
    with torch.cuda.device(buf.device):
        _check(L.bm_decompress(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.c_void_p(out.data_ptr()),
                               _stream(stream)))
    return out


def coeff_count(shape, block=17, levels=2, global_levels=2, rounds=1) -> int:
    n = ctypes.c_size_t(0)
    p = _params(block, levels, global_levels, rounds=rounds)
    _check(load().bm_coeff_count(len(shape), _shape(shape), ctypes.byref(p), ctypes.byref(n)))
    return n.value


def decompose(field: torch.Tensor, block=17, levels=2, global_levels=2, stream=None, rounds=1) -> torch.Tensor:
    """Full-precision multilevel coefficients in stream order."""
    _dev_check(field)
    n = coeff_count(field.shape, block, levels, global_levels, rounds)
    out = torch.empty(n, dtype=field.dtype, device=field.device)
    p = _params(block, levels, global_levels, rounds=rounds)
    with torch.cuda.device(field.device):
        _check(load().bm_decompose(ctypes.c_void_p(field.data_ptr()), field.dim(), _shape(field.shape), _dtype(field.dtype),
                                   ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def recompose(coeffs: torch.Tensor, shape, block=17, levels=2, global_levels=2, stream=None,
              rounds=1) -> torch.Tensor:
    _dev_check(coeffs)
    out = torch.empty(tuple(shape), dtype=coeffs.dtype, device=coeffs.device)
    p = _params(block, levels, global_levels, rounds=rounds)
    with torch.cuda.device(coeffs.device):
        _check(load().bm_recompose(ctypes.c_void_p(coeffs.data_ptr()), len(shape), _shape(shape), _dtype(coeffs.dtype),
                                   ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def decompose_adjoint(coeff_grad: torch.Tensor, shape, block=17, levels=2, global_levels=2,
                      stream=None) -> torch.Tensor:
    """Transpose of :func:`decompose` applied to coefficient gradients: the
    gradient with respect to the field (the field's shape)."""
    _dev_check(coeff_grad)
    if coeff_grad.numel() != coeff_count(shape, block, levels, global_levels):
        raise ValueError("coefficient gradient has the wrong length")
    out = torch.empty(tuple(shape), dtype=coeff_grad.dtype, device=coeff_grad.device)
    p = _params(block, levels, global_levels)
    with torch.cuda.device(coeff_grad.device):
        _check(load().bm_decompose_adjoint(ctypes.c_void_p(coeff_grad.data_ptr()), len(shape), _shape(shape),
                                           _dtype(coeff_grad.dtype), ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                           _stream(stream)))
    return out


def recompose_adjoint(field_grad: torch.Tensor, block=17, levels=2, global_levels=2, stream=None) -> torch.Tensor:
    """Transpose of :func:`recompose` applied to field gradients: the gradient
    with respect to the coefficients (stream order)."""
    _dev_check(field_grad)
    n = coeff_count(field_grad.shape, block, levels, global_levels)
    out = torch.empty(n, dtype=field_grad.dtype, device=field_grad.device)
    p = _params(block, levels, global_levels)
    with torch.cuda.device(field_grad.device):
        _check(load().bm_recompose_adjoint(ctypes.c_void_p(field_grad.data_ptr()), field_grad.dim(), _shape(field_grad.shape),
                                           _dtype(field_grad.dtype), ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                           _stream(stream)))
    return out


class Decompose(torch.autograd.Function):
    """Differentiable decomposition: backward is the transposed operator (no
    saved tensors: the operator is linear)."""

    @staticmethod
    def forward(ctx, field, block=17, levels=2, global_levels=2):
        ctx.params = (tuple(field.shape), block, levels, global_levels)
        return decompose(field.contiguous(), block, levels, global_levels)

    @staticmethod
    def backward(ctx, g):
        shape, block, levels, global_levels = ctx.params
        return decompose_adjoint(g.contiguous(), shape, block, levels, global_levels), None, None, None


class Recompose(torch.autograd.Function):
    """Differentiable recomposition: backward is the transposed operator."""

    @staticmethod
    def forward(ctx, coeffs, shape, block=17, levels=2, global_levels=2):
        ctx.params = (block, levels, global_levels)
        return recompose(coeffs.contiguous(), shape, block, levels, global_levels)

    @staticmethod
    def backward(ctx, g):
        block, levels, global_levels = ctx.params
        return recompose_adjoint(g.contiguous(), block, levels, global_levels), None, None, None, None


def decompose_ad(field, block=17, levels=2, global_levels=2):
    return Decompose.apply(field, block, levels, global_levels)


def recompose_ad(coeffs, shape, block=17, levels=2, global_levels=2):
    return Recompose.apply(coeffs, tuple(int(v) for v in shape), block, levels, global_levels)


def stream_codes(buf: torch.Tensor, stream=None) -> torch.Tensor:
    _dev_check(buf)
    info = stream_info(buf)
    out = torch.empty(info["n_coeffs"], dtype=torch.int32, device=buf.device)
    with torch.cuda.device(buf.device):
        _check(load().bm_stream_codes(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.c_void_p(out.data_ptr()),
                                      _stream(stream)))
    return out


def huffman_encode(symbols: torch.Tensor, dict_size: int, chunk: int = 2048, stream=None):
    """Huffman section of int16/uint16 symbols; returns (uint8 tensor, sizes)."""
    _dev_check(symbols)
    if symbols.element_size() != 2:
        raise TypeError("symbols must be a 16-bit tensor")
    n = symbols.numel()
    nch = (n + chunk - 1) // chunk
    cap = 64 + 8 * nch + 2 * dict_size + 16 * 1024 + 4 * n + 8 * nch
    out = torch.empty(cap, dtype=torch.uint8, device=symbols.device)
    sizes = (ctypes.c_uint64 * 5)()
    with torch.cuda.device(symbols.device):
        _check(load().bm_huffman_encode(ctypes.c_void_p(symbols.data_ptr()), n, int(dict_size), int(chunk),
                                        ctypes.c_void_p(out.data_ptr()), cap, sizes, _stream(stream)))
    s = [int(v) for v in sizes]
    meta = {"codebook_bytes": s[0], "n_runs": s[1], "n_chunks": s[2], "n_words": s[3], "bytes": s[4]}
    return out[: s[4]], meta


def huffman_decode(section: torch.Tensor, meta: dict, n: int, dict_size: int, chunk: int = 2048, stream=None):
    _dev_check(section)
    out = torch.empty(n, dtype=torch.int16, device=section.device)
    sizes = (ctypes.c_uint64 * 5)(meta["codebook_bytes"], meta["n_runs"], meta["n_chunks"], meta["n_words"],
                                  meta["bytes"])
    with torch.cuda.device(section.device):
        _check(load().bm_huffman_decode(ctypes.c_void_p(section.data_ptr()), sizes, n, int(dict_size), int(chunk),
                                        ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def set_timing(enabled: bool):
    load().bm_set_timing(1 if enabled else 0)


def stage_timeline() -> list:
    """(name, start_ms, ms) of every stage of the last timed call."""
    L = load()
    names = (ctypes.c_char_p * 64)()
    ms = (ctypes.c_float * 64)()
    t0 = (ctypes.c_float * 64)()
    n = L.bm_stage_timeline(names, ms, t0, 64)
    return [(names[i].decode(), float(t0[i]), float(ms[i])) for i in range(n)]


def stage_times() -> list:
    L = load()
    names = (ctypes.c_char_p * 64)()
    ms = (ctypes.c_float * 64)()
    n = L.bm_stage_times(names, ms, 64)
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def set_block_grid_limit(max_ctas: int):
    """Cap the persistent grid of the In-cache Block kernels (0 = default)."""
    load().bm_set_block_grid_limit(int(max_ctas))


def launch_count() -> int:
    return int(load().bm_launch_count())


def release_workspace(stream=None):
    load().bm_release_workspace(None if stream is None else ctypes.c_void_p(stream.cuda_stream))
