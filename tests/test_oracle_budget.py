"""Pins of the oracle's error control (Sec. II-B level shares, Sec. III-C ROI
tolerances, tau_global = min_i tau_i) and of its quantiser, by brute force and
closed forms."""
import numpy as np
import pytest

import fields
import oracle


def _recompose_matrix(shape, B, K, M):
    p = oracle.plan(shape, B, K, M)
    cols = []
    for j in range(p["n_coeffs"]):
        e = np.zeros(p["n_coeffs"])
        e[j] = 1.0
        cols.append(oracle.recompose(e, shape, B, K, M).ravel())
    return np.stack(cols, axis=1), p


def _local_counts(B, K):
    """Detail counts of the K levels inside one B^3 block (n -> n//2+1)."""
    out, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        out.append(n ** 3 - c ** 3)
        n = c
    return out


def _q_per_coeff(p, B, K, M, q, ntiers=1, block_tier=None):
    parts = []
    for b in range(p["nblocks"]):
        t = 0 if block_tier is None else int(block_tier[b])
        parts += [np.full(c, q[t * K + l]) for l, c in enumerate(_local_counts(B, K))]
    parts += [np.full(c, q[ntiers * K + l]) for l, c in enumerate(p["global_counts"])]
    parts.append(np.full(p["coarsest"], q[ntiers * K + M]))
    return np.concatenate(parts)


@pytest.mark.parametrize("shape,B,K,M", [
    ((9, 9, 9), 9, 2, 0),
    ((9, 9, 9), 9, 1, 1),
    ((18, 9, 9), 9, 1, 1),
    ((8, 8, 16), 8, 1, 1),
])
def test_linf_bound_brute_force(shape, B, K, M):
    """Worst-case reconstruction error sum_j |A_ij| * q_j/2 over every output
    node, with A the assembled recomposition matrix, stays within tau."""
    A, p = _recompose_matrix(shape, B, K, M)
    tau = 1.0
    q, margin, raw = oracle.budget(shape, B, K, M, [tau], 0.0, True)
    assert margin == 0.0 and not raw
    delta = _q_per_coeff(p, B, K, M, q) / 2.0
    worst = np.abs(A) @ delta
    assert worst.max() <= tau * (1 + 1e-12)
    # the split is not vacuous: the bound uses a sizeable part of the budget
    assert worst.max() >= 0.2 * tau


def test_budget_shares_closed_form():
    """N = K + M detail levels plus the coarsest array share tau' equally;
    detail level l gets tau'/((N+1) A_l), the coarsest tau'/(N+1); global
    levels and the coarsest use the strictest tier (tau_global = min_i tau_i)."""
    shape, B, K, M = (36, 36, 36), 9, 2, 2
    A = oracle.level_constants(shape, B, K, M)
    q, margin, raw = oracle.budget(shape, B, K, M, [2.0e-3, 5.0e-2], 10.0, False)
    N = K + M
    eps32 = 2.0 ** -24
    assert margin == pytest.approx(8 * eps32 * (N + 1) * 10.0, rel=1e-15)
    taup = np.array([2.0e-3, 5.0e-2]) - margin
    for t in range(2):
        for l in range(K):
            assert q[t * K + l] == pytest.approx(2 * taup[t] / ((N + 1) * A[l]), rel=1e-15)
    for l in range(M):
        assert q[2 * K + l] == pytest.approx(2 * taup[0] / ((N + 1) * A[K + l]), rel=1e-15)
    assert q[2 * K + M] == pytest.approx(2 * taup[0] / (N + 1), rel=1e-15)
    assert not raw


def _level_error_matrix(shape, B, K, M, level):
    """Dense map from one level's coefficients to the reconstructed field, all
    other coefficients zero (columns = unit coefficient vectors)."""
    p = oracle.plan(shape, B, K, M)
    if level < K:  # local level of block 0: its coefficients come after the finer levels
        start = sum(_local_counts(B, K)[:level])
        count = _local_counts(B, K)[level]
    else:
        start = p["nblocks"] * p["per_block"] + sum(p["global_counts"][: level - K])
        count = p["global_counts"][level - K]
    cols = []
    for j in range(start, start + count):
        e = np.zeros(p["n_coeffs"])
        e[j] = 1.0
        cols.append(oracle.recompose(e, shape, B, K, M).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("shape,B,K,M,level", [
    ((9, 9, 9), 9, 1, 0, 0),
    ((8, 8, 8), 8, 1, 0, 0),
    ((5, 5, 5), 5, 1, 0, 0),
    ((9, 9, 9), 9, 2, 0, 1),
    ((10, 8, 12), 2, 0, 1, 0),
    ((18, 9, 9), 9, 1, 1, 1),
])
def test_level_constant_is_exact_error_operator_norm(shape, B, K, M, level):
    """A_l equals the max row abs sum of the dense error operator of level l,
    assembled by recomposing unit coefficient vectors.  When finer levels
    follow, the level's error passes through their interpolation, which copies
    coarse nodes and averages at fine ones, so the max row sum is unchanged."""
    A = oracle.level_constants(shape, B, K, M)[level]
    R = _level_error_matrix(shape, B, K, M, level)
    exact = np.abs(R).sum(axis=1).max()
    assert exact <= A <= exact + 1.5 / 65536


def test_margin_forces_raw_when_tolerance_near_roundoff():
    shape, B, K, M = (18, 18, 18), 9, 1, 1
    # FP32: margin = 8 * 2^-24 * 3 * max|u|; tau below twice that -> raw
    m = 8 * 2.0 ** -24 * 3 * 1.0
    _, margin, raw = oracle.budget(shape, B, K, M, [1.9 * m], 1.0, False)
    assert raw and margin == pytest.approx(m)
    _, _, raw = oracle.budget(shape, B, K, M, [2.1 * m], 1.0, False)
    assert not raw


@pytest.mark.parametrize("f64", [False, True])
def test_quantizer_special_cases(f64):
    q = 0.25  # power of two: c/q exact
    for k in range(-5, 6):
        assert oracle.quantize(k * q, q, f64) == (k, False)
        assert oracle.quantize((k + 0.5) * q, q, f64) == (k + 1, False)  # ties go up
    assert oracle.quantize(0.0, q, f64) == (0, False)
    assert oracle.quantize(-0.0, q, f64) == (0, False)
    _, ov = oracle.quantize(2.0 ** 31 * q, q, f64)
    assert ov
    _, ov = oracle.quantize(np.nan, q, f64)
    assert ov


@pytest.mark.parametrize("f64", [False, True])
def test_quantizer_is_round_half_up(f64):
    rng = np.random.default_rng(11)
    q = 3.7e-3
    c = rng.normal(0, 5.0, 20000)
    if not f64:
        c = c.astype(np.float32).astype(np.float64)
    exact = c / q + 0.5
    want = np.floor(exact)
    rel = 1e-6 if not f64 else 1e-13
    near = np.abs(exact - np.rint(exact)) < rel * np.maximum(1, np.abs(exact))
    got = np.array([oracle.quantize(v, q, f64)[0] for v in c])
    assert np.all(got[~near] == want[~near])
    assert np.all(np.abs(got[near] - want[near]) <= 1)


@pytest.mark.parametrize("f64", [False, True])
def test_quantizer_array_is_round_half_up(f64):
    """The element-wise quantiser: floor(c/q + 1/2) away from bin edges (the
    rounding decision in the field's precision may differ by one bin only
    next to an edge), per-element widths, overflow flags for huge and NaN
    values."""
    rng = np.random.default_rng(12)
    c = rng.normal(0, 3.0, 30000)
    q = 10.0 ** rng.uniform(-4, -1, c.size)
    if not f64:
        c = c.astype(np.float32).astype(np.float64)
    exact = c / q + 0.5
    rel = 1e-6 if not f64 else 1e-13
    near = np.abs(exact - np.rint(exact)) < rel * np.maximum(1, np.abs(exact))
    big = np.abs(exact) >= 2.0 ** 30
    codes, ovf = oracle.quantize_array(c, q, f64)
    ok = ~near & ~big
    assert np.all(codes[ok] == np.floor(exact[ok]))
    assert np.all(np.abs(codes[near & ~big] - np.floor(exact[near & ~big])) <= 1)
    assert np.all(ovf == big)
    _, ov = oracle.quantize_array(np.array([np.nan, 2.0 ** 40, -(2.0 ** 40), 0.0]), 1.0, f64)
    assert list(ov) == [True, True, True, False]


def test_bound_holds_end_to_end_with_roi():
    """Per-region L-inf: ROI blocks at tau 1e-5, background 1e-2 (relative)."""
    u = fields.roi_field((40, 37, 29), seed=4).numpy()
    B, K, M = 9, 2, 1
    roi_mask = fields.gradient_roi(u, B)
    roi = np.where(roi_mask, 1e-5, 1e-2)
    s = oracle.compress(u, 1e-2, rel=True, roi=roi, B=B, K=K, M=M)
    d = oracle.decompress(s)
    err = np.abs(d - u)
    mx = np.abs(u).max()
    tau_node = np.repeat(np.repeat(np.repeat(roi, B, 0), B, 1), B, 2)[: u.shape[0], : u.shape[1], : u.shape[2]] * mx
    assert np.all(err <= tau_node)
    assert roi_mask.any() and (~roi_mask).any()
