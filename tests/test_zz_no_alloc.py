"""bm_huffman_encode_noalloc: the Huffman encoder for callers that cannot
allocate device memory (a process whose device memory another allocator
reserved up front, or a loop that cannot take the device-wide synchronisation
of cudaMalloc/cudaFree).  Its scratch is a static device array shared by
every call, so it must give the same bytes as bm_huffman_encode on
consecutive calls, each one clearing what the previous call left behind, and
it must leave the device's free memory unchanged.  Kept in a file collected
last."""
import ctypes

import numpy as np
import pytest
import torch

import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as bm

    L = bm.load()
    for name in ("bm_huffman_encode", "bm_huffman_encode_noalloc"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                      ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
        f.restype = ctypes.c_int
    return L


def _encode(fn, sym, dict_size, chunk):
    t = torch.from_numpy(sym.view(np.int16)).to("cuda:0")
    cap = 64 + 16 * sym.size + 4 * dict_size + 16 * (sym.size // chunk + 2)
    out = torch.full((cap,), 0xAB, dtype=torch.uint8, device="cuda:0")
    sizes = (ctypes.c_uint64 * 5)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(ctypes.c_void_p(t.data_ptr()), sym.size, dict_size, chunk, ctypes.c_void_p(out.data_ptr()), cap, sizes,
            stream)
    assert st == 0
    torch.cuda.synchronize()
    return out[: sizes[4]].cpu().numpy(), [int(v) for v in sizes]


def test_noalloc_matches_allocating_encoder_twice(lib):
    cases = [
        (fields.laplace_symbols(1_000_003, 4096, 40.0, seed=31), 8192, 2048),
        (fields.laplace_symbols(250_000, 512, 0.4, seed=32, escape_rate=0.002), 1024, 1024),
    ]
    for sym, dict_size, chunk in cases:  # two calls in a row, different inputs
        want, wsz = _encode(lib.bm_huffman_encode, sym, dict_size, chunk)
        got, gsz = _encode(lib.bm_huffman_encode_noalloc, sym, dict_size, chunk)
        assert gsz == wsz
        np.testing.assert_array_equal(got, want)


def test_noalloc_allocates_nothing(lib):
    """After one warm-up call (which may load kernels), further calls leave
    the device's free memory exactly where it was."""
    sym = fields.laplace_symbols(400_000, 2048, 12.0, seed=33)
    dict_size, chunk = 4096, 2048
    t = torch.from_numpy(sym.view(np.int16)).to("cuda:0")
    cap = 64 + 16 * sym.size + 4 * dict_size + 16 * (sym.size // chunk + 2)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda:0")
    sizes = (ctypes.c_uint64 * 5)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        st = lib.bm_huffman_encode_noalloc(ctypes.c_void_p(t.data_ptr()), sym.size, dict_size, chunk,
                                           ctypes.c_void_p(out.data_ptr()), cap, sizes, stream)
        assert st == 0

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_capturing_stream(lib):
    """The call synchronises, which graph capture forbids: it refuses a
    capturing stream without enqueuing anything, and the capture stays valid."""
    sym = fields.laplace_symbols(10_000, 256, 3.0, seed=34)
    t = torch.from_numpy(sym.view(np.int16)).to("cuda:0")
    out = torch.empty(1 << 20, dtype=torch.uint8, device="cuda:0")
    x = torch.zeros(4, device="cuda:0")
    sizes = (ctypes.c_uint64 * 5)()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        x.add_(1.0)
        st = lib.bm_huffman_encode_noalloc(ctypes.c_void_p(t.data_ptr()), sym.size, 512, 256,
                                           ctypes.c_void_p(out.data_ptr()), out.numel(), sizes,
                                           ctypes.c_void_p(s.cuda_stream))
        g.capture_end()
    assert st == 1
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0


def test_noalloc_rejects_requests_beyond_its_scratch(lib):
    sym = np.zeros(16384 * 64 + 1, dtype=np.uint16)
    t = torch.from_numpy(sym.view(np.int16)).to("cuda:0")
    out = torch.empty(1 << 22, dtype=torch.uint8, device="cuda:0")
    sizes = (ctypes.c_uint64 * 5)()
    st = lib.bm_huffman_encode_noalloc(ctypes.c_void_p(t.data_ptr()), sym.size, 64, 64,
                                       ctypes.c_void_p(out.data_ptr()), out.numel(), sizes, None)
    assert st == 1
