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


def test_batched_kernel_groups_and_fallbacks(bm):
    """A batch mixing every kind of item: groups of the persistent forward
    kernel (FP32 B17 K2, FP32 B9 K1, FP64 B9 K2 with a ROI map, FP64 B17 K1,
    a field of ~7 M elements spanning many max|u| slices), and items that keep
    their own pipeline (a planar field, B = 8, two rounds), a field with a NaN
    (raw stream) and one with an infinity; every stream equals the single
    call's byte for byte, and two items match the oracle."""
    rng = np.random.default_rng(7)
    specs = [
        ((200, 190, 180), torch.float32, dict(block=17, levels=2, global_levels=2), 1e-3),
        ((45, 38, 52), torch.float32, dict(block=17, levels=2, global_levels=2), 1e-4),
        ((30, 70, 41), torch.float32, dict(block=17, levels=2, global_levels=1), 1e-2),
        ((40, 33, 29), torch.float32, dict(block=9, levels=1, global_levels=1), 5e-3),
        ((27, 30, 36), torch.float32, dict(block=9, levels=1, global_levels=2), 1e-5),
        ((41, 37, 33), torch.float64, dict(block=9, levels=2, global_levels=2), 1e-4),
        ((25, 31, 29), torch.float64, dict(block=9, levels=2, global_levels=2), 2e-3),
        ((35, 18, 40), torch.float64, dict(block=17, levels=1, global_levels=1), 1e-6),
        ((300, 257), torch.float32, dict(block=17, levels=2, global_levels=2), 1e-3),
        ((40, 37, 45), torch.float32, dict(block=8, levels=2, global_levels=1), 1e-3),
        ((70, 61, 53), torch.float32, dict(block=17, levels=2, global_levels=1, rounds=2), 1e-3),
        ((33, 34, 35), torch.float32, dict(block=17, levels=2, global_levels=2), 1e-3),
        ((34, 35, 36), torch.float32, dict(block=17, levels=2, global_levels=2), 1e-3),
    ]
    fs, tols, rois, params = [], [], [], []
    for i, (shape, dt, p, tol) in enumerate(specs):
        u = fields.power_law_grf(shape, exponent=-3.0, seed=500 + i, dtype=dt, device=DEV).contiguous()
        fs.append(u)
        tols.append(tol)
        params.append(p)
        roi = None
        if i == 5:
            nb = int(np.prod([(s + p["block"] - 1) // p["block"] for s in shape]))
            roi = np.full(nb, tol)
            roi[rng.choice(nb, size=max(1, nb // 8), replace=False)] = tol / 10
        rois.append(roi)
    fs[11].view(-1)[12345] = float("nan")
    fs[12].view(-1)[777] = float("inf")
    out = bm.compress_batch(fs, tols, rois=rois, params=params)
    for i, (u, t, r, p, s) in enumerate(zip(fs, tols, rois, params, out)):
        ref = bm.compress(u, t, roi=r, **p)
        assert torch.equal(s, ref), i
    for i in (1, 5):
        u = fs[i].cpu().numpy()
        p = params[i]
        check_stream_parity(bm, u, out[i].cpu().numpy(), tols[i], "rel", p["block"], p["levels"], p["global_levels"],
                            roi=rois[i], label="batched_kernel_item%d" % i, dev=DEV)
    # the same batch again: the second call is captured as a CUDA graph, the
    # third and fourth replay it (tickets and flags start afresh each time)
    for _ in range(3):
        again = bm.compress_batch(fs, tols, rois=rois, params=params)
        for a, b in zip(out, again):
            assert torch.equal(a, b)
    # new field values under the same arguments: the replayed graph reads them
    for u in fs[:11]:
        u.mul_(0.5).add_(0.25)
    out2 = bm.compress_batch(fs, tols, rois=rois, params=params)
    for i, (u, t, r, p, s) in enumerate(zip(fs, tols, rois, params, out2)):
        assert torch.equal(s, bm.compress(u, t, roi=r, **p)), i
    # other arguments (a tolerance, a ROI entry): not the captured graph
    tols2 = list(tols)
    tols2[3] = 2e-3
    rois2 = [None if r is None else r.copy() for r in rois]
    rois2[5][0] = tols[5] / 100
    for _ in range(3):
        out3 = bm.compress_batch(fs, tols2, rois=rois2, params=params)
        for i, (u, t, r, p, s) in enumerate(zip(fs, tols2, rois2, params, out3)):
            assert torch.equal(s, bm.compress(u, t, roi=r, **p)), i
