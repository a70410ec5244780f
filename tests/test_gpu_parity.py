"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (per the workload statement): coefficients within 1e-5 (FP32) / 1e-12
(FP64) of max|u|; codes identical except +-1 flips explained by a coefficient
sitting within the coefficient tolerance of a bin edge, counted inside and
outside the 1e-6 relative window and recorded; the hard gate: the oracle's
quantiser on the GPU's own coefficients gives the GPU's codes exactly; Huffman
codebook and bitstream bit-exact given identical symbols; the L-inf bound
holds at every node of every region.
"""
import numpy as np
import pytest
import torch

import fields
import oracle

from _util import check_stream_parity, per_block_tau, q_per_coeff

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (name, shape, dtype, B, K, M): sizes the oracle finishes in seconds, spanning
# several blocks with ragged tails
CASES = [
    ("bumps65_b9k3", (65, 65, 65), np.float32, 9, 3, 0),
    ("grf_b17k2m2", (70, 61, 53), np.float32, 17, 2, 2),
    ("grf_b9k1m3", (37, 29, 44), np.float32, 9, 1, 3),
    ("roi_f64_b9k2m2", (47, 41, 33), np.float64, 9, 2, 2),
    ("f64_b17k3m1", (35, 18, 40), np.float64, 17, 3, 1),
    ("tiny_2x3x2", (2, 3, 2), np.float32, 9, 1, 1),
    # gathered grids with lines of more than 1087 nodes (the dense projection
    # path of the global levels), along dimension 0 and along dimension 2
    ("long0_b9k1m1", (2000, 6, 5), np.float32, 9, 1, 1),
    ("long2_f64_b9k1m1", (5, 6, 2000), np.float64, 9, 1, 1),
    # block sizes without a fused block kernel (the paper's 8-node blocks,
    # 16 and 33 nodes): the in-cache levels as blocked whole-grid passes
    ("grf_b8k3m1", (40, 37, 45), np.float32, 8, 3, 1),
    ("roi_f64_b8k1m2", (47, 41, 33), np.float64, 8, 1, 2),
    ("grf_b16k2m2", (70, 61, 53), np.float32, 16, 2, 2),
    ("grf_b33k2m1", (70, 40, 66), np.float32, 33, 2, 1),
]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    return m


def _field(name, shape, dtype):
    if name.startswith("bumps"):
        u = fields.gaussian_bumps(shape, seed=1)
    elif name.startswith("roi"):
        u = fields.roi_field(shape, seed=3).numpy()
    else:
        u = fields.power_law_grf(shape, seed=2).numpy()
    return np.ascontiguousarray(u.astype(dtype))


def _coef_tol(u):
    return (1e-5 if u.dtype == np.float32 else 1e-12) * float(np.abs(u).max())


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_decompose_matches_oracle(bm, case):
    name, shape, dt, B, K, M = case
    u = _field(name, shape, dt)
    g = bm.decompose(torch.from_numpy(u).to(DEV), block=B, levels=K, global_levels=M).cpu().numpy()
    o = oracle.decompose(u.astype(np.float64), B, K, M)
    assert g.shape == o.shape
    err = np.abs(g.astype(np.float64) - o).max()
    assert err <= _coef_tol(u), err


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_recompose_matches_oracle(bm, case):
    """GPU recomposition of the oracle's coefficients equals the oracle's."""
    name, shape, dt, B, K, M = case
    u = _field(name, shape, dt)
    o = oracle.decompose(u.astype(np.float64), B, K, M)
    g = bm.recompose(torch.from_numpy(o.astype(dt)).to(DEV), shape, block=B, levels=K, global_levels=M).cpu().numpy()
    r = oracle.recompose(o.astype(dt).astype(np.float64), shape, B, K, M)
    assert np.abs(g.astype(np.float64) - r).max() <= 4 * _coef_tol(u)
    # and it inverts the decomposition
    assert np.abs(g.astype(np.float64) - u).max() <= 8 * _coef_tol(u)


def _check_compress_parity(bm, u, tol, mode, B, K, M, roi=None, label="", radius=32768):
    t = torch.from_numpy(u).to(DEV)
    sg = bm.compress(t, tol, mode=mode, roi=roi, block=B, levels=K, global_levels=M, radius=radius).cpu().numpy()
    return check_stream_parity(bm, u, sg, tol, mode, B, K, M, roi=roi, label=label, dev=DEV, radius=radius)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_compress_parity(bm, case, tol):
    name, shape, dt, B, K, M = case
    u = _field(name, shape, dt)
    roi = None
    if name.startswith("roi"):
        mask = fields.gradient_roi(u, B)
        roi = np.where(mask, tol * 1e-2, tol)
    _check_compress_parity(bm, u, tol, "rel", B, K, M, roi=roi, label=name)


def _smooth_with_spikes(shape, dtype):
    """A smooth field with a few large spikes: small codes almost everywhere,
    escapes near the spikes, and codes beyond 16 bits at the spikes."""
    i, j, k = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    u = np.sin(0.05 * i) * np.cos(0.04 * j) + 0.5 * np.sin(0.03 * k)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, u.size, 30)
    u.ravel()[idx] += rng.choice([-1.0, 1.0], 30) * 3.0
    return np.ascontiguousarray(u.astype(dtype))


@pytest.mark.parametrize("radius", [4096, 32768])
@pytest.mark.parametrize("dt,B,K,M", [(np.float32, 17, 2, 2), (np.float32, 9, 3, 1), (np.float64, 9, 2, 2)])
def test_wide_code_parity(bm, dt, B, K, M, radius):
    """Escapes in groups with and without codes beyond 16 bits (the block
    kernels stage codes in 16 bits and send wider ones straight to the escape
    array), against the oracle, with a small dictionary (escapes below 2^15)
    and the full 16-bit one."""
    u = _smooth_with_spikes((40, 37, 45), dt)
    co = _check_compress_parity(bm, u, 1e-4, "abs", B, K, M, label="spikes_r%d" % radius, radius=radius)
    assert co is not None
    assert int((np.abs(co) >= 32768).sum()) > 0
    assert int(((np.abs(co) >= radius) & (np.abs(co) < 32767)).sum()) > 0 or radius == 32768
    assert int(((np.abs(co) >= 4096) & (np.abs(co) < 32767)).sum()) > 0


@pytest.mark.parametrize("radius", [4096, 32768])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_codes_at_the_dictionary_edge(bm, dt, radius):
    """Codes exactly at and around the largest 16-bit symbol: isolated spikes
    on level-one detail nodes (all coarse neighbours zero, so the coefficient
    is the spike itself) sized to give codes of +-(2^15 - 2) .. +-(2^15 + 1)
    and far beyond; the stream must match the oracle's (code 2^15 - 1 is
    symbol 2^16 - 1 with the full dictionary, code 2^15 escapes)."""
    B, K, M = 9, 1, 0
    shape = (36, 27, 27)
    tol = 1e-3
    u = np.zeros(shape, dtype=np.float64)
    targets = [32766, 32767, 32768, 32769, -32766, -32767, -32768, -32769, 40000, -100000, 5, -7]
    # the widths depend on max|u| through the round-off margin: iterate to the fixed point
    q, _, _ = oracle.budget(shape, B, K, M, [tol], 1.0, dt == np.float64)
    for _ in range(5):
        q, _, _ = oracle.budget(shape, B, K, M, [tol], float(dt(100000 * q[0])), dt == np.float64)
    for i, code in enumerate(targets):  # node (1,1,1) of block i along dims 0..2
        b0, b1 = divmod(i, 3)
        u[9 * b0 + 1, 9 * b1 + 1, 1] = code * q[0]
    u = np.ascontiguousarray(u.astype(dt))
    co = _check_compress_parity(bm, u, tol, "abs", B, K, M, label="edge_r%d" % radius, radius=radius)
    assert co is not None
    for code in targets:
        assert code in set(int(c) for c in co), code


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gpu_decodes_oracle_stream(bm, case):
    """The GPU decoder reproduces the oracle's decompression of the oracle's stream."""
    name, shape, dt, B, K, M = case
    u = _field(name, shape, dt)
    so = oracle.compress(u, 1e-3, rel=True, B=B, K=K, M=M)
    do = oracle.decompress(so).astype(np.float64)
    st = torch.from_numpy(so).to(DEV)
    dg = bm.decompress(st).cpu().numpy().astype(np.float64)
    assert np.abs(dg - do).max() <= 8 * _coef_tol(u)
    if not oracle.stream_header(so)["raw"]:
        _, codes = oracle.decompress(so, want_codes=True)
        np.testing.assert_array_equal(bm.stream_codes(st).cpu().numpy(), codes)


@pytest.mark.parametrize("scale,esc,chunk,dict_size", [
    (0.3, 0.0, 2048, 8192), (5.0, 0.001, 1024, 8192), (300.0, 0.01, 1536, 8192), (0.0, 0.0, 64, 64),
    (40.0, 0.0, 256, 1024), (2000.0, 0.0, 2048, 8192),
    # the full 16-bit dictionary: present symbols within the encoder's window
    # and the shared-memory codebook, spread over more than the window, and so
    # many that the codebook and decoder tables take global scratch
    (200.0, 0.002, 2048, 65536), (1500.0, 0.0, 1024, 65536), (6000.0, 0.001, 2048, 65536),
    (30000.0, 0.0, 512, 65536),
])
def test_huffman_bit_exact(bm, scale, esc, chunk, dict_size):
    sym = fields.laplace_symbols(300_007, dict_size // 2, scale, seed=17, escape_rate=esc)
    so, mo = oracle.huffman_encode(sym, dict_size, chunk)
    t = torch.from_numpy(sym.view(np.int16)).to(DEV)
    sg, mg = bm.huffman_encode(t, dict_size, chunk)
    assert mg == mo
    np.testing.assert_array_equal(sg.cpu().numpy(), so)
    back = bm.huffman_decode(sg, mg, sym.size, dict_size, chunk).cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(back, sym)


@pytest.mark.parametrize("dict_size,chunk", [(64, 2048), (65536, 1024)])
def test_huffman_codes_up_to_32_bits(bm, dict_size, chunk):
    """Fibonacci counts (1, 1, 2, 3, 5, ...) over 33 symbols make the most
    skewed Huffman tree: codes of 1 to 32 bits.  The encoder keeps a code of
    at most 26 bits and its length in one table word; the longer ones (the
    seven rarest symbols here, a 32-bit code among them) come from the full
    code table.  A 64-symbol dictionary takes the shared-memory table, the
    16-bit one the global table; 9,227,464 symbols in shuffled order end in a
    ragged chunk."""
    fib = [1, 1]
    while len(fib) < 33:
        fib.append(fib[-1] + fib[-2])
    rng = np.random.default_rng(5)
    present = rng.choice(np.arange(dict_size), size=33, replace=False)
    sym = np.repeat(present, fib).astype(np.uint16)
    rng.shuffle(sym)
    f = np.bincount(sym, minlength=dict_size)
    L = oracle.huffman_lengths(f)
    assert L.max() == 32 and (L > 26).sum() == 7
    so, mo = oracle.huffman_encode(sym, dict_size, chunk)
    t = torch.from_numpy(sym.view(np.int16)).to(DEV)
    sg, mg = bm.huffman_encode(t, dict_size, chunk)
    assert mg == mo
    np.testing.assert_array_equal(sg.cpu().numpy(), so)
    back = bm.huffman_decode(sg, mg, sym.size, dict_size, chunk).cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(back, sym)


def _table_mode(codes, radius=32768):
    """The encoder's table for a call's codes, by the rule its codebook
    applies: 0 when the present symbols span fewer than 8192, 3 fewer than
    57344, 1 when the 57344 symbols centred on code 0 (and the escape symbol)
    hold at least half of them and escapes fewer than a fifth, else 2."""
    sym = np.where(np.abs(codes) < radius, codes + radius, 0)
    f = np.bincount(sym.astype(np.int64), minlength=2 * radius)
    present = np.flatnonzero(f)
    span = present.max() - present.min()
    lo = radius - 57344 // 2
    win = f[lo:lo + 57344].sum() + f[0]
    if span < 8192:
        return 0
    if span < 57344:
        return 3
    return 1 if 2 * win >= f.sum() and 5 * f[0] < f.sum() else 2


@pytest.mark.parametrize("tol,mode", [(1e-2, 0), (1e-3, 3), (1e-4, 1), (3e-5, 2)])
def test_encoder_table_modes(bm, tol, mode):
    """One compress call per table of the encoder: the same 64^3 GRF at four
    tolerances spans about 2,200 symbols (the small shared-memory window),
    22,000 (the large window), the whole dictionary with a few symbols outside
    the large window (looked up in the global table) and 1 % escapes, and the
    whole dictionary with 27 % escapes (the global table); every stream is
    Huffman-coded, none a raw copy."""
    shape = (64, 64, 64)
    u = fields.power_law_grf(shape, seed=7, dtype=torch.float32).numpy()
    so, codes = oracle.compress(u, tol, rel=True, B=9, K=2, M=2, want_codes=True)
    assert _table_mode(codes) == mode and not oracle.stream_header(so)["raw"]
    sg = bm.compress(torch.from_numpy(u).to(DEV), tol, block=9, levels=2, global_levels=2).cpu().numpy()
    check_stream_parity(bm, u, sg, tol, "rel", 9, 2, 2, label=f"encoder_mode{mode}")


def test_huffman_heavy_tails(bm):
    """Two symbols far out in the tails of a 65,536-symbol dictionary (outside
    the wide histogram's 49,152 shared-memory bins, so counted with global
    atomics) with 6 M occurrences each beside a Laplace centre: counts, code
    lengths and the stream must be the oracle's byte for byte."""
    rng = np.random.default_rng(23)
    centre = fields.laplace_symbols(1_200_003, 32768, 40.0, seed=29, escape_rate=0.0)
    sym = np.concatenate([centre, np.full(6_000_000, 7, np.uint16), np.full(6_000_000, 61_000, np.uint16)])
    rng.shuffle(sym)
    so, mo = oracle.huffman_encode(sym, 65536, 2048)
    sg, mg = bm.huffman_encode(torch.from_numpy(sym.view(np.int16)).to(DEV), 65536, 2048)
    assert mg == mo
    np.testing.assert_array_equal(sg.cpu().numpy(), so)


def test_huffman_single_symbol(bm):
    sym = np.full(5000, 77, dtype=np.uint16)
    so, mo = oracle.huffman_encode(sym, 128, 256)
    sg, mg = bm.huffman_encode(torch.from_numpy(sym.view(np.int16)).to(DEV), 128, 256)
    assert mg == mo
    np.testing.assert_array_equal(sg.cpu().numpy(), so)


def test_raw_fallbacks(bm):
    u = fields.gaussian_bumps((20, 21, 22), seed=4)
    u[3, 4, 5] = np.nan
    sg = bm.compress(torch.from_numpy(u).to(DEV), 1e-2, block=9, levels=2, global_levels=1).cpu().numpy()
    np.testing.assert_array_equal(sg, oracle.compress(u, 1e-2, rel=True, B=9, K=2, M=1))
    d = bm.decompress(torch.from_numpy(sg).to(DEV)).cpu().numpy()
    np.testing.assert_array_equal(d.view(np.uint32), u.view(np.uint32))
    w = fields.gaussian_bumps((20, 21, 22), seed=4)
    w[1, 2, 3] = -np.inf
    sg = bm.compress(torch.from_numpy(w).to(DEV), 1e-2, block=9, levels=2, global_levels=1).cpu().numpy()
    np.testing.assert_array_equal(sg, oracle.compress(w, 1e-2, rel=True, B=9, K=2, M=1))
    v = fields.gaussian_bumps((20, 21, 22), seed=4)
    sg = bm.compress(torch.from_numpy(v).to(DEV), 1e-7, block=9, levels=2, global_levels=1).cpu().numpy()
    assert oracle.stream_header(sg)["raw"]
    np.testing.assert_array_equal(sg, oracle.compress(v, 1e-7, rel=True, B=9, K=2, M=1))


def test_corrupt_streams_rejected(bm):
    u = fields.gaussian_bumps((30, 30, 30), seed=5)
    s = bm.compress(torch.from_numpy(u).to(DEV), 1e-3, block=9, levels=2, global_levels=1)
    good = s.clone()
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.decompress(good[:-8].clone())
    assert e.value.status == 4
    bad = good.clone()
    bad[0] ^= 0x55
    with pytest.raises(bm.BlockMGARDError):
        bm.decompress(bad)
    # chunk word counts no longer add up to the bitstream length
    h = oracle.stream_header(good.cpu().numpy())
    bad = good.clone()
    bad[h["off_chunks"]] = (int(bad[h["off_chunks"]]) + 1) % 256
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.decompress(bad)
    assert e.value.status == 4
    # random bit flips inside the bitstream: either detected or decoded, never a fault
    rng = np.random.default_rng(0)
    for _ in range(5):
        bad = good.clone()
        pos = int(rng.integers(h["off_bits"], h["total"]))
        bad[pos] ^= 0x10
        try:
            bm.decompress(bad)
        except bm.BlockMGARDError as err:
            assert err.status == 4
    torch.cuda.synchronize()
    # the context is still usable
    d = bm.decompress(good).cpu().numpy()
    assert np.abs(d - u).max() <= 1e-3 * np.abs(u).max()


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[0]], ids=["grf_b17k2m2", "roi_f64_b9k2m2", "bumps65_b9k3"])
def test_several_blocks_per_cta(bm, case):
    """Every CTA walks several blocks (capped persistent grid): same streams and
    coefficients as the oracle, and the GPU round trip within the bound."""
    name, shape, dt, B, K, M = case
    u = _field(name, shape, dt)
    t = torch.from_numpy(u).to(DEV)
    ref = {tol: bm.compress(t, tol, mode="rel", block=B, levels=K, global_levels=M).cpu().numpy() for tol in (1e-2, 1e-4)}
    try:
        bm.set_block_grid_limit(3)
        g = bm.decompose(t, block=B, levels=K, global_levels=M).cpu().numpy()
        o = oracle.decompose(u.astype(np.float64), B, K, M)
        assert np.abs(g.astype(np.float64) - o).max() <= _coef_tol(u)
        r = bm.recompose(torch.from_numpy(g).to(DEV), shape, block=B, levels=K, global_levels=M).cpu().numpy()
        assert np.abs(r.astype(np.float64) - u).max() <= 8 * _coef_tol(u)
        for tol in (1e-2, 1e-4):
            sg = bm.compress(t, tol, mode="rel", block=B, levels=K, global_levels=M).cpu().numpy()
            np.testing.assert_array_equal(sg, ref[tol])  # independent of the grid
            d = bm.decompress(torch.from_numpy(sg).to(DEV)).cpu().numpy().astype(np.float64)
            assert np.abs(d - u).max() <= tol * np.abs(u).max()
    finally:
        bm.set_block_grid_limit(0)


def test_overflow_gives_raw(bm):
    """Values near the FP32 maximum overflow the FP32 interpolation (the FP64
    oracle does not): the stream must fall back to an exact raw copy."""
    u = np.full((20, 21, 22), 3.0e38, dtype=np.float32)
    u[3, 4, 5] = 2.9e38
    sg = bm.compress(torch.from_numpy(u).to(DEV), 1e-2, mode="rel", block=9, levels=2, global_levels=1)
    assert oracle.stream_header(sg.cpu().numpy())["raw"]
    d = bm.decompress(sg).cpu().numpy()
    np.testing.assert_array_equal(d.view(np.uint32), u.view(np.uint32))


def test_invalid_arguments(bm):
    t = torch.zeros((10, 10, 10), device=DEV)
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.compress(t, -1.0)
    assert e.value.status == 1
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.compress(t, 1e-3, block=2)
    assert e.value.status == 1
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.compress(t, 1e-3, block=65)
    assert e.value.status == 1
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.recompose_adjoint(t, block=8, levels=1, global_levels=1)
    assert e.value.status == 5
    with pytest.raises(bm.BlockMGARDError):
        bm.compress(t, 1e-3, block=9, levels=4)
    with pytest.raises(bm.BlockMGARDError):
        bm.compress(t, 1e-3, chunk=100)
    with pytest.raises(bm.BlockMGARDError):
        bm.compress(t, 1e-3, chunk=4096)
