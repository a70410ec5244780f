"""1-D and 2-D fields through the C ABI against the oracle.  A dimension of
extent 1 is neither blocked nor coarsened; the library runs the in-cache
levels of such fields on the block-major grid of their blocks.  Checked:
coefficients and recomposition against the oracle, streams (tiers, q table,
codes with explained flips only, the hard gate, byte-identical when no code
flips), the L-inf bound at every node of every region, the GPU decoding the
oracle's streams, and explicit extents of 1 anywhere in a 3-D shape."""
import numpy as np
import pytest
import torch

import fields
import oracle

from _util import check_stream_parity, coef_tol

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (name, shape, dtype, B, K, M): ragged tails, several blocks, both dtypes
CASES = [
    ("line_f32_b17k2m2", (3500,), np.float32, 17, 2, 2),
    ("line_f64_b9k3m1", (3001,), np.float64, 9, 3, 1),
    ("line_f32_b9k1m0", (1234,), np.float32, 9, 1, 0),
    ("plane_f32_b17k2m2", (300, 211), np.float32, 17, 2, 2),
    ("plane_f64_b9k2m1", (97, 130), np.float64, 9, 2, 1),
    ("plane_f32_b9k3m2", (64, 65), np.float32, 9, 3, 2),
    ("plane_f32_tiny", (2, 3), np.float32, 9, 1, 1),
]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


def _field(shape, dtype, seed=11):
    if len(shape) == 2:
        u = fields.power_law_grf((1,) + tuple(shape), exponent=-2.0, seed=seed).numpy().reshape(shape)
    else:
        u = np.cumsum(np.random.default_rng(seed).normal(size=shape)) * 0.01
    return np.ascontiguousarray(u.astype(dtype))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_lowdim_decompose_recompose(bm, case):
    name, shape, dt, B, K, M = case
    u = _field(shape, dt)
    g = bm.decompose(torch.from_numpy(u).to(DEV), block=B, levels=K, global_levels=M).cpu().numpy()
    o = oracle.decompose(u.astype(np.float64), B, K, M)
    assert g.shape == o.shape
    assert np.abs(g.astype(np.float64) - o).max() <= coef_tol(u)
    r = bm.recompose(torch.from_numpy(o.astype(dt)).to(DEV), shape, block=B, levels=K, global_levels=M).cpu().numpy()
    assert r.shape == u.shape
    ro = oracle.recompose(o.astype(dt).astype(np.float64), shape, B, K, M)
    assert np.abs(r.astype(np.float64) - ro).max() <= 4 * coef_tol(u)
    assert np.abs(r.astype(np.float64) - u).max() <= 8 * coef_tol(u)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_lowdim_compress_parity(bm, case, tol):
    name, shape, dt, B, K, M = case
    u = _field(shape, dt)
    roi = None
    if len(shape) == 2 and min(shape) > B:
        nb = int(np.prod([-(-s // B) for s in shape]))
        roi = np.where(np.random.default_rng(2).random(nb) < 0.25, tol / 30, tol)
    t = torch.from_numpy(u).to(DEV)
    sg = bm.compress(t, tol, mode="rel", roi=roi, block=B, levels=K, global_levels=M).cpu().numpy()
    assert oracle.stream_header(sg)["ndim"] == len(shape)
    check_stream_parity(bm, u, sg, tol, "rel", B, K, M, roi=roi, label=name, dev=DEV)
    d = bm.decompress(torch.from_numpy(sg).to(DEV))
    assert tuple(d.shape) == tuple(shape)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_lowdim_gpu_decodes_oracle_stream(bm, case):
    name, shape, dt, B, K, M = case
    u = _field(shape, dt)
    so = oracle.compress(u, 1e-3, rel=True, B=B, K=K, M=M)
    do = oracle.decompress(so).astype(np.float64)
    dg = bm.decompress(torch.from_numpy(so).to(DEV)).cpu().numpy().astype(np.float64)
    assert dg.shape == do.shape
    assert np.abs(dg - do).max() <= 8 * coef_tol(u)


@pytest.mark.parametrize("shape3,shape", [((1, 40, 23), (40, 23)), ((40, 1, 23), (40, 23)), ((1, 1, 700), (700,)),
                                          ((700, 1, 1), (700,))])
def test_unit_extents_anywhere(bm, shape3, shape):
    """The same values with an explicit extent of 1 anywhere in a 3-D shape
    give the same coefficients as the 1-D / 2-D field, on the GPU and in the
    oracle."""
    u = _field(shape, np.float32)
    t2 = torch.from_numpy(u).to(DEV)
    t3 = t2.reshape(shape3)
    c2 = bm.decompose(t2, block=9, levels=2, global_levels=1).cpu().numpy()
    c3 = bm.decompose(t3, block=9, levels=2, global_levels=1).cpu().numpy()
    np.testing.assert_array_equal(c2, c3)
    np.testing.assert_allclose(c3, oracle.decompose(u.reshape(shape3).astype(np.float64), 9, 2, 1),
                               atol=coef_tol(u), rtol=0)
    s3 = bm.compress(t3, 1e-3, block=9, levels=2, global_levels=1)
    d = bm.decompress(s3)
    assert tuple(d.shape) == shape3
    assert float((d - t3).abs().max()) <= 1e-3 * float(t3.abs().max())


def test_lowdim_batch_and_unsupported(bm):
    """2-D and 1-D items in a batch give the single calls' streams; re-blocking
    rounds and the adjoints refuse fields with extents of 1."""
    us = [torch.from_numpy(_field((250, 180), np.float32, 1)).to(DEV),
          torch.from_numpy(_field((5000,), np.float64, 2)).to(DEV),
          torch.from_numpy(_field((40, 50, 30), np.float32, 3)).to(DEV)]
    tols = [1e-3, 1e-4, 1e-2]
    out = bm.compress_batch(us, tols, block=9, levels=2, global_levels=2)
    for u, tol, s in zip(us, tols, out):
        assert torch.equal(s, bm.compress(u, tol, block=9, levels=2, global_levels=2))
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.compress(us[0], 1e-3, block=9, levels=1, global_levels=1, rounds=2)
    assert e.value.status in (1, 5)
    with pytest.raises(bm.BlockMGARDError) as e:
        bm.recompose_adjoint(us[0], block=9, levels=1, global_levels=1)
    assert e.value.status == 5
