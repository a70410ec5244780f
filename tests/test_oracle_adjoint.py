"""The transposed operators the adjoint kernels implement, pinned on the CPU.

The decomposition level is D = (Id - I R_C) u at the non all-coarse nodes and
c = R_C u + P D (Sec. II-B).  Its transpose, for gradients (g_D, g_c), is
g_u = v + R_C^T (g_c - I^T v) with v = S_F^T g_D + P^T g_c; the
recomposition's transpose is g_c = I^T g, g_D = S_F (g - P^T g_c).  Both
formulas, written with the independent quadrature-built 1-D operators of the
operator tests, must equal the transpose of the oracle's operator assembled
column by column; the assembled operators must also invert each other.
"""
import numpy as np
import pytest

import oracle

from test_oracle_operators import _kron3, independent_1d


def _level_pieces(n):
    C, I, Mf, Mc, P = independent_1d(np.arange(n, dtype=float))
    nc = len(C)
    S = np.zeros((nc, n))
    S[np.arange(nc), C] = 1.0
    S3, I3, P3 = _kron3(S, S, S), _kron3(I, I, I), _kron3(P, P, P)
    coarse = np.zeros(n ** 3, dtype=bool)
    coarse[S3.argmax(axis=1)] = True
    SF = np.eye(n ** 3)[~coarse]
    return S3, I3, P3, SF


@pytest.mark.parametrize("n", [5, 9])
def test_decompose_transpose_formula(n):
    S3, I3, P3, SF = _level_pieces(n)
    nd = SF.shape[0]
    rng = np.random.default_rng(n)
    gD, gc = rng.standard_normal(nd), rng.standard_normal(S3.shape[0])
    v = SF.T @ gD + P3.T @ gc
    formula = v + S3.T @ (gc - I3.T @ v)
    A = oracle.decompose_matrix((n, n, n), n, 1, 0)
    np.testing.assert_allclose(A.T @ np.concatenate([gD, gc]), formula.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(oracle.decompose_adjoint(np.concatenate([gD, gc]), (n, n, n), n, 1, 0).ravel(),
                               formula, atol=1e-12)


@pytest.mark.parametrize("n", [5, 9])
def test_recompose_transpose_formula(n):
    S3, I3, P3, SF = _level_pieces(n)
    rng = np.random.default_rng(10 + n)
    g = rng.standard_normal(n ** 3)
    gc = I3.T @ g
    gD = SF @ (g - P3.T @ gc)
    got = oracle.recompose_adjoint(g.reshape(n, n, n), (n, n, n), n, 1, 0)
    np.testing.assert_allclose(got, np.concatenate([gD, gc]), atol=1e-12)


@pytest.mark.parametrize("shape,B,K,M", [((11, 10, 12), 9, 2, 1), ((9, 9, 19), 9, 1, 2)])
def test_assembled_operators_invert_each_other(shape, B, K, M):
    A = oracle.decompose_matrix(shape, B, K, M)
    R = oracle.recompose_matrix(shape, B, K, M)
    np.testing.assert_allclose(R @ A, np.eye(A.shape[1]), atol=1e-11)
