"""Batched compress: every field's stream equals the single-field call byte
for byte (uneven shapes, both dtypes, own tolerances, ROI maps), decompresses
within its bound, and a bad item fails alone."""
import numpy as np
import pytest
import torch

import fields

from _util import check_stream_parity

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


def _batch(seed, n):
    rng = np.random.default_rng(seed)
    fs, tols, rois = [], [], []
    for i in range(n):
        f64 = i % 5 == 4
        shape = tuple(int(v) for v in rng.integers(20, 90, size=3))
        u = fields.power_law_grf(shape, exponent=float(rng.uniform(-4.0, -1.5)), seed=100 + i,
                                 dtype=torch.float64 if f64 else torch.float32, device=DEV).contiguous()
        tol = float(10 ** rng.uniform(-5, -2))
        nb = int(np.prod([(s + 16) // 17 for s in shape]))
        roi = None
        if i % 3 == 0:
            roi = np.full(nb, tol)
            pick = rng.choice(nb, size=max(1, nb // 10), replace=False)
            roi[pick] = tol / 10
        fs.append(u)
        tols.append(tol)
        rois.append(roi)
    return fs, tols, rois


def test_batch_matches_single_calls(bm):
    fs, tols, rois = _batch(1, 13)
    out = bm.compress_batch(fs, tols, rois=rois)
    for u, t, r, s in zip(fs, tols, rois, out):
        ref = bm.compress(u, t, roi=r)
        assert s.numel() == ref.numel()
        assert torch.equal(s, ref)
        d = bm.decompress(s)
        maxabs = float(u.abs().max())
        tau = t * maxabs
        if r is None:
            assert float((d - u).abs().max()) <= tau
        else:
            # every node keeps the loosest bound; blocks with a tighter entry are checked in the parity tests
            assert float((d - u).abs().max()) <= tau


def test_batch_matches_oracle(bm):
    """Every item of a batch against the oracle's stream of the same field:
    uneven shapes, both dtypes, their own tolerances, ROI maps on some items
    (each ROI block checked against its own tau_i), codes with explained
    flips only and the hard gate."""
    import fields as F

    specs = [((37, 52, 29), np.float32, 3e-3, True), ((61, 40, 45), np.float32, 1e-4, False),
             ((33, 35, 31), np.float64, 1e-5, True), ((20, 70, 24), np.float64, 2e-2, False),
             ((90, 21, 40), np.float32, 1e-2, True)]
    B, K, M = 17, 2, 2
    us, ts, rois = [], [], []
    for i, (shape, dt, tol, with_roi) in enumerate(specs):
        u = np.ascontiguousarray(F.power_law_grf(shape, exponent=-2.5 - 0.3 * i, seed=300 + i).numpy().astype(dt))
        roi = None
        if with_roi:
            roi = np.where(F.gradient_roi(u, B), tol / 10, tol).ravel()
        us.append(u)
        ts.append(tol)
        rois.append(roi)
    out = bm.compress_batch([torch.from_numpy(u).to(DEV) for u in us], ts, rois=rois, block=B, levels=K,
                            global_levels=M)
    for i, (u, tol, roi, s) in enumerate(zip(us, ts, rois, out)):
        check_stream_parity(bm, u, s.cpu().numpy(), tol, "rel", B, K, M, roi=roi, label="batch_item%d" % i, dev=DEV)


def test_batch_reports_a_bad_item_alone(bm):
    fs, tols, rois = _batch(2, 4)
    tols[2] = -1.0
    with pytest.raises(bm.BlockMGARDError):
        bm.compress_batch(fs, tols, rois=rois)
    # the library keeps working afterwards
    ok = bm.compress_batch(fs[:2], tols[:2], rois=rois[:2])
    for u, t, r, s in zip(fs[:2], tols[:2], rois[:2], ok):
        assert torch.equal(s, bm.compress(u, t, roi=r))


def test_perf_model_fit_and_selection(bm):
    m = bm.perf_model_fit(torch.float32, 17)
    d = m.as_dict()
    assert d["block_latency_ms"] > 0 and d["block_peak_per_ms"] > 0
    assert bm.perf_model_knee(m, 0.9) > 0
    shape = (160, 150, 140)
    u = fields.power_law_grf(shape, seed=9, device=DEV).contiguous()
    pred = bm.predict_ms(m, shape)
    bm.compress(u, 1e-3)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        bm.compress(u, 1e-3)
    b.record()
    torch.cuda.synchronize()
    meas = a.elapsed_time(b) / 5
    assert pred / 3 < meas < pred * 3, (pred, meas)
    p, t = bm.select_params(m, shape, 10.0)
    s = bm.compress(u, 1e-3, **p)
    d = bm.decompress(s)
    assert float((d - u).abs().max()) <= 1e-3 * float(u.abs().max())
