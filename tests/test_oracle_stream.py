"""Oracle stream round trips: L-inf per region, header fields, raw fallback."""
import numpy as np
import pytest

import fields
import oracle


@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-4])
def test_fp32_bumps_roundtrip(tol):
    u = fields.gaussian_bumps((30, 33, 28), seed=1)
    rng = float(u.max() - u.min())
    s = oracle.compress(u, tol * rng, rel=False, B=9, K=3, M=0)
    h = oracle.stream_header(s)
    assert h["total"] == s.size
    if tol >= 1e-3:
        assert not h["raw"]
    elif h["raw"]:  # noise-dominated at this tolerance: raw copy when not smaller
        assert s.size == 256 + u.nbytes
    d = oracle.decompress(s)
    assert d.dtype == np.float32
    assert np.abs(d.astype(np.float64) - u).max() <= tol * rng


@pytest.mark.parametrize("B,K,M", [(17, 2, 2), (16, 2, 1), (8, 1, 2), (9, 2, 2)])
def test_grf_hybrid_roundtrip(B, K, M):
    u = fields.power_law_grf((41, 37, 45), seed=2).numpy()
    for rel in [1e-2, 1e-4]:
        s, codes = oracle.compress(u, rel, rel=True, B=B, K=K, M=M, want_codes=True)
        d, dcodes = oracle.decompress(s, want_codes=True)
        assert np.abs(d.astype(np.float64) - u).max() <= rel * np.abs(u).max()
        if not oracle.stream_header(s)["raw"]:
            np.testing.assert_array_equal(codes, dcodes)


def test_outliers_present_and_decoded():
    """A small dictionary (radius 64) on a smooth FP64 field: coarse-level codes
    exceed it and go to the outlier section, which decoding restores."""
    u = fields.gaussian_bumps((36, 36, 36), seed=5, noise=0.0).astype(np.float64)
    s, codes = oracle.compress(u, 1e-3, rel=True, B=9, K=1, M=1, radius=64, want_codes=True)
    h = oracle.stream_header(s)
    assert not h["raw"]
    assert h["n_outliers"] > 0
    assert h["n_outliers"] == int(np.sum(np.abs(codes) >= 64))
    d, dcodes = oracle.decompress(s, want_codes=True)
    np.testing.assert_array_equal(codes, dcodes)
    assert np.abs(d - u).max() <= 1e-3 * np.abs(u).max()


def test_raw_fallback_nonfinite_and_tight():
    u = fields.gaussian_bumps((12, 12, 12), seed=2)
    u[3, 4, 5] = np.nan
    s = oracle.compress(u, 1e-2, rel=True, B=9, K=1, M=0)
    h = oracle.stream_header(s)
    assert h["raw"] and s.size == 256 + u.nbytes
    d = oracle.decompress(s)
    np.testing.assert_array_equal(d.view(np.uint32), u.view(np.uint32))
    v = fields.gaussian_bumps((12, 12, 12), seed=2)
    s = oracle.compress(v, 1e-7, rel=True, B=9, K=1, M=0)  # below FP32 round-off margin
    assert oracle.stream_header(s)["raw"]


def test_fp64_tiers_header():
    u = fields.roi_field((20, 20, 20), seed=6).numpy()
    roi = np.full((3, 3, 3), 1e-2)
    roi[1, 1, 1] = 1e-5
    roi[0, 2, 1] = 1e-4
    s = oracle.compress(u, 1e-2, rel=True, roi=roi, B=7, K=1, M=1)
    h = oracle.stream_header(s)
    assert h["f64"] and h["n_tiers"] == 3
    tiers = s[h["off_tiers"]:h["off_tiers"] + 24].view(np.float64)
    np.testing.assert_allclose(tiers, np.array([1e-5, 1e-4, 1e-2]) * np.abs(u).max(), rtol=1e-15)
    d = oracle.decompress(s)
    err = np.abs(d - u)
    mx = np.abs(u).max()
    assert err[7:14, 7:14, 7:14].max() <= 1e-5 * mx
    assert err.max() <= 1e-2 * mx
