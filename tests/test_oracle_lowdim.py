"""Pins of the oracle on 1-D and 2-D fields.  A field of fewer than three
dimensions is held as a 3-D field with leading extents of 1; a dimension of
extent 1 is neither blocked nor coarsened (its one-node level operator is the
identity), so the transform is the tensor product of the 1-D operators over
the remaining dimensions (Sec. II-B), applied per block (Sec. III-A).

Checked against facts that do not come from the oracle: Kronecker assembly of
independently built 1-D operators (hats and Gauss quadrature), linear and
bilinear fields giving zero coefficients, the equivalence of explicit unit
dimensions anywhere in a 3-D shape, brute-force L-inf bounds over assembled
recomposition matrices, and the level constants as exact operator norms."""
import numpy as np
import pytest

import fields
import oracle

from test_oracle_operators import independent_1d


def _one_level_2d(n):
    """One level on one n x n block: [coefficients at non-coarse nodes
    (row-major), corrected coarse values (row-major)] from independent 1-D
    operators, assembled with np.kron."""
    C, I, Mf, Mc, P = independent_1d(np.arange(n, dtype=float))
    nc = len(C)
    S = np.zeros((nc, n))
    S[np.arange(nc), C] = 1.0
    S2, I2, P2 = np.kron(S, S), np.kron(I, I), np.kron(P, P)
    Dmap = np.eye(n * n) - I2 @ S2
    coarse = np.zeros(n * n, dtype=bool)
    coarse[S2.argmax(axis=1)] = True
    return np.vstack([Dmap[~coarse], S2 + P2 @ Dmap])


@pytest.mark.parametrize("n", [5, 9])
def test_2d_operator_equals_kronecker_assembly(n):
    A = _one_level_2d(n)
    O = np.stack([oracle.decompose(np.eye(n * n)[j].reshape(n, n), n, 1, 0) for j in range(n * n)], axis=1)
    assert O.shape == A.shape
    np.testing.assert_allclose(O, A, atol=1e-13)


@pytest.mark.parametrize("n", [5, 9, 17])
def test_1d_operator_is_the_1d_level(n):
    C, I, Mf, Mc, P = independent_1d(np.arange(n, dtype=float))
    S = np.zeros((len(C), n))
    S[np.arange(len(C)), C] = 1.0
    Dmap = np.eye(n) - I @ S
    fine = np.setdiff1d(np.arange(n), C)
    A = np.vstack([Dmap[fine], S + P @ Dmap])
    O = np.stack([oracle.decompose(np.eye(n)[j], n, 1, 0) for j in range(n)], axis=1)
    np.testing.assert_allclose(O, A, atol=1e-13)


def _multilinear(shape):
    axes = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    u = 0.3 + sum((d + 1) * 0.7 * a for d, a in enumerate(axes))
    if len(shape) == 2:
        u = u - 0.05 * axes[0] * axes[1]
    return u


@pytest.mark.parametrize("shape,B,K,M", [
    ((36,), 9, 2, 2), ((64,), 16, 2, 1), ((34,), 17, 1, 2),
    ((18, 27), 9, 2, 2), ((32, 16), 8, 2, 1), ((34, 17), 17, 1, 2),
])
def test_linear_fields_have_zero_coefficients(shape, B, K, M):
    u = _multilinear(shape)
    c = oracle.decompose(u, B, K, M)
    p = oracle.plan(shape, B, K, M)
    assert np.abs(c[: p["n_coeffs"] - p["coarsest"]]).max() <= 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("shape,B,K,M,R", [
    ((100,), 9, 2, 2, 1), ((1000,), 17, 2, 3, 1), ((77,), 8, 2, 1, 1), ((300,), 9, 1, 1, 2),
    ((40, 23), 9, 2, 1, 1), ((33, 65), 17, 2, 2, 1), ((20, 21), 8, 1, 2, 1), ((50, 31), 9, 1, 1, 2),
    ((2, 2), 9, 1, 1, 1), ((3,), 9, 1, 0, 1),
])
def test_recompose_inverts_decompose_lowdim(shape, B, K, M, R):
    u = np.random.default_rng(3).normal(size=shape)
    c = oracle.decompose(u, B, K, M, R)
    assert c.size == oracle.plan(shape, B, K, M, R)["n_coeffs"]
    r = oracle.recompose(c, shape, B, K, M, R)
    assert r.shape == u.shape
    assert np.abs(r - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("shape3,shape", [
    ((1, 40, 23), (40, 23)), ((40, 1, 23), (40, 23)), ((40, 23, 1), (40, 23)),
    ((1, 1, 70), (70,)), ((70, 1, 1), (70,)), ((1, 70, 1), (70,)),
])
def test_unit_dimensions_anywhere_are_not_blocked(shape3, shape):
    """The same values held with an explicit extent-1 dimension at any
    position: identical coefficients, plan and stream (stream up to the
    recorded number of dimensions)."""
    u = np.random.default_rng(4).normal(size=shape)
    for B, K, M in ((9, 2, 1), (17, 1, 2)):
        np.testing.assert_array_equal(oracle.decompose(u.reshape(shape3), B, K, M), oracle.decompose(u, B, K, M))
        s2 = oracle.compress(u, 1e-3, B=B, K=K, M=M)
        s3 = oracle.compress(u.reshape(shape3), 1e-3, B=B, K=K, M=M)
        if shape3[0] == 1 and (len(shape) == 2 or shape3[1] == 1):  # same 3-D layout of the shape
            h2 = oracle.stream_header(s2)
            assert h2["ndim"] == len(shape) and oracle.stream_header(s3)["ndim"] == 3
            np.testing.assert_array_equal(np.delete(s2, np.s_[8:12]), np.delete(s3, np.s_[8:12]))


def _recompose_matrix(shape, B, K, M):
    p = oracle.plan(shape, B, K, M)
    A = np.stack([oracle.recompose(np.eye(p["n_coeffs"])[j], shape, B, K, M).ravel()
                  for j in range(p["n_coeffs"])], axis=1)
    return A, p


def _level_counts(p_per_block_dims, B, K):
    out, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        out.append(n ** p_per_block_dims - c ** p_per_block_dims)
        n = c
    return out


@pytest.mark.parametrize("shape,B,K,M", [((18, 9), 9, 1, 1), ((9, 9), 9, 2, 0), ((27,), 9, 2, 1), ((16, 8), 8, 1, 1)])
def test_linf_bound_brute_force_lowdim(shape, B, K, M):
    A, p = _recompose_matrix(shape, B, K, M)
    q, margin, raw = oracle.budget(shape, B, K, M, [1.0], 0.0, True)
    assert margin == 0.0 and not raw
    parts = []
    for _ in range(p["nblocks"]):
        parts += [np.full(c, q[l]) for l, c in enumerate(_level_counts(len(shape), B, K))]
    parts += [np.full(c, q[K + l]) for l, c in enumerate(p["global_counts"])]
    parts.append(np.full(p["coarsest"], q[K + M]))
    delta = np.concatenate(parts) / 2.0
    worst = np.abs(A) @ delta
    assert worst.max() <= 1.0 + 1e-12
    assert worst.max() >= 0.2


@pytest.mark.parametrize("shape,B", [((9, 9), 9), ((8, 8), 8), ((17,), 17), ((9,), 9)])
def test_level_constant_is_exact_norm_lowdim(shape, B):
    """A_1 of a one-block 1-D / 2-D level equals the max row abs sum of the
    dense map from its coefficients to the reconstructed field."""
    A1 = oracle.level_constants(shape, B, 1, 0)[0]
    p = oracle.plan(shape, B, 1, 0)
    cnt = p["n_coeffs"] - p["coarsest"]
    R = np.stack([oracle.recompose(np.eye(p["n_coeffs"])[j], shape, B, 1, 0).ravel() for j in range(cnt)], axis=1)
    exact = np.abs(R).sum(axis=1).max()
    assert exact <= A1 <= exact + 1.5 / 65536
    # a 2-D level is not a 3-D one: its constant differs from the cube's
    if len(shape) == 2:
        assert A1 != oracle.level_constants((B, B, B), B, 1, 0)[0]


@pytest.mark.parametrize("shape,B,K,M,dt", [
    ((5000,), 17, 2, 2, np.float32), ((777,), 9, 1, 3, np.float64),
    ((300, 211), 17, 2, 2, np.float32), ((97, 130), 9, 2, 1, np.float64),
])
def test_bound_end_to_end_lowdim(shape, B, K, M, dt):
    """Compress / decompress 1-D and 2-D fields with a ROI map: every node
    within its block's tolerance, the field's own dimensions restored."""
    rng = np.random.default_rng(5)
    u = np.cumsum(rng.normal(size=shape), axis=-1).astype(dt)
    nb = int(np.prod([-(-s // B) for s in shape]))
    roi = np.where(rng.random(nb) < 0.2, 1e-5, 1e-3)
    s = oracle.compress(u, 1e-3, rel=True, roi=roi, B=B, K=K, M=M)
    d = oracle.decompress(s)
    assert d.shape == u.shape and d.dtype == u.dtype
    tau = roi.reshape([-(-n // B) for n in shape]) * np.abs(u).max()
    for ax in range(len(shape)):
        tau = np.repeat(tau, B, axis=ax)
    tau = tau[tuple(slice(0, n) for n in shape)]
    assert np.all(np.abs(d.astype(np.float64) - u) <= tau)
