"""Pins of the oracle's decomposition (Sec. II-B / III-A of the paper) against
facts that do not come from the oracle itself:

* the printed worked facts of the 8^3 block (Sec. III-A, III-D);
* a closed form (L2 projection of a hat onto P1 is a constant);
* operators assembled independently here: hat functions evaluated directly
  and mass matrices by Gauss quadrature, combined with ``np.kron``;
* invariants: multilinear fields have zero coefficients; recompose inverts
  decompose.
"""
import os

import numpy as np
import pytest

import fields
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------------------
# independent 1-D construction (no oracle code): hats + quadrature
# ---------------------------------------------------------------------------
def _coarse_set(n):
    return sorted(set(range(0, n, 2)) | {n - 1})


def _hat(nodes, j, t):
    e = np.zeros(len(nodes))
    e[j] = 1.0
    return np.interp(t, nodes, e)


def _gauss_points(x):
    """2-point Gauss-Legendre nodes/weights on every cell of x (exact for the
    piecewise quadratic products of hats)."""
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    pts, wts = [], []
    for a, b in zip(x[:-1], x[1:]):
        mid, half = 0.5 * (a + b), 0.5 * (b - a)
        pts.extend(mid + half * g)
        wts.extend([half, half])
    return np.array(pts), np.array(wts)


def independent_1d(x):
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    C = _coarse_set(n)
    xc = x[C]
    t, w = _gauss_points(x)
    phi_f = np.stack([_hat(x, j, t) for j in range(n)])          # n x q
    phi_c = np.stack([_hat(xc, J, t) for J in range(len(C))])     # nc x q
    Mf = (phi_f * w) @ phi_f.T
    Mc = (phi_c * w) @ phi_c.T
    I = np.stack([_hat(xc, J, x) for J in range(len(C))], axis=1)  # n x nc
    # L2 projection of sum_i D_i phi_i onto span(phi_c): Mc z = (phi_c, phi_f) D
    G = (phi_c * w) @ phi_f.T
    P = np.linalg.solve(Mc, G)
    return C, I, Mf, Mc, P


# ---------------------------------------------------------------------------
def test_closed_form_hat_projection():
    for row in _rows("closed_form_hat.txt"):
        xs, d, z = [p.split() for p in row.split("|")]
        x = np.array([float(v) for v in xs])
        _, _, _, P = oracle.level_1d(x)
        got = P @ np.array([0.0, float(d[0]), 0.0])
        np.testing.assert_allclose(got, [float(v) for v in z], rtol=0, atol=1e-15)


def test_block8_structure_matches_paper():
    g = dict(r.split(None, 1) for r in _rows("block8_structure.txt"))
    n = int(g["block_nodes"])
    I, Mf, Mc, P = oracle.level_1d(np.arange(n))
    nc = P.shape[0]
    assert nc == int(g["coarse_nodes"])
    # coarse set of 8 nodes: even indices plus the last one
    coarse_rows = [i for i in range(n) if np.count_nonzero(I[i]) == 1 and I[i].max() == 1.0]
    assert coarse_rows == [0, 2, 4, 6, 7]
    shapes = [(n, n, n), (nc, n, n), (nc, nc, n), (nc, nc, nc)]
    assert " ".join("x".join(map(str, s)) for s in shapes) == g["pass_shapes"]
    total = sum(int(np.prod(s)) for s in shapes)
    assert total == int(g["working_set_elements"])
    assert 4 * total == int(g["working_set_bytes_fp32"])
    assert 8 * total == int(g["working_set_bytes_fp64"])
    p = oracle.plan((8, 8, 8), 8, 1, 0)
    assert p["per_block"] == int(g["detail_values"])
    assert p["m"] ** 3 == int(g["coarse_values"])


@pytest.mark.parametrize("n", list(range(2, 41)))
def test_coarsening_count(n):
    I, _, _, P = oracle.level_1d(np.arange(n, dtype=float))
    assert P.shape[0] == n // 2 + 1


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("n", [3, 4, 5, 8, 9, 16, 17, 30])
def test_1d_operators_vs_quadrature(n, seed):
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.uniform(0.2, 3.0, size=n))
    C, I, Mf, Mc, P = independent_1d(x)
    oI, oMf, oMc, oP = oracle.level_1d(x)
    np.testing.assert_allclose(oI, I, atol=1e-14)
    np.testing.assert_allclose(oMf, Mf, atol=1e-13 * x[-1])
    np.testing.assert_allclose(oMc, Mc, atol=1e-13 * x[-1])
    np.testing.assert_allclose(oP, P, atol=1e-11)


def _kron3(a, b, c):
    return np.kron(a, np.kron(b, c))


def _dense_level_operator(n):
    """Full one-level map u (n^3) -> [coefficients at non-coarse nodes
    (row-major), corrected coarse values (row-major)] from the independent
    1-D operators."""
    C, I, Mf, Mc, P = independent_1d(np.arange(n, dtype=float))
    nc = len(C)
    S = np.zeros((nc, n))
    S[np.arange(nc), C] = 1.0
    S3 = _kron3(S, S, S)
    I3 = _kron3(I, I, I)
    P3 = _kron3(P, P, P)
    Dmap = np.eye(n ** 3) - I3 @ S3
    coarse_mask = np.zeros(n ** 3, dtype=bool)
    coarse_mask[S3.argmax(axis=1)] = True
    detail_rows = Dmap[~coarse_mask]
    coarse_rows = S3 + P3 @ Dmap
    return np.vstack([detail_rows, coarse_rows])


@pytest.mark.parametrize("n", [5, 9])
def test_3d_operator_equals_kronecker_assembly(n):
    A = _dense_level_operator(n)
    # oracle's operator, column by column
    cols = []
    for j in range(n ** 3):
        e = np.zeros(n ** 3)
        e[j] = 1.0
        cols.append(oracle.decompose(e.reshape(n, n, n), n, 1, 0))
    O = np.stack(cols, axis=1)
    assert O.shape == A.shape
    np.testing.assert_allclose(O, A, atol=1e-13)


@pytest.mark.parametrize("shape,B,K,M", [
    ((18, 27, 36), 9, 2, 2),
    ((16, 32, 16), 8, 2, 1),
    ((34, 17, 17), 17, 1, 2),
    ((32, 16, 48), 16, 2, 2),
    ((27, 27, 27), 9, 3, 1),
])
def test_multilinear_has_zero_coefficients(shape, B, K, M):
    u = fields.smooth_multilinear(shape)
    c = oracle.decompose(u, B, K, M)
    p = oracle.plan(shape, B, K, M)
    details = c[: p["n_coeffs"] - p["coarsest"]]
    assert np.abs(details).max() <= 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("shape,B,K,M", [
    ((20, 23, 17), 9, 2, 1),
    ((20, 23, 17), 8, 2, 2),
    ((33, 47, 65), 17, 2, 2),
    ((33, 47, 65), 16, 1, 3),
    ((10, 11, 12), 9, 3, 0),
    ((5, 5, 5), 5, 1, 0),
])
def test_recompose_inverts_decompose(shape, B, K, M):
    u = fields.gaussian_bumps(shape, seed=7).astype(np.float64)
    c = oracle.decompose(u, B, K, M)
    assert c.size == oracle.plan(shape, B, K, M)["n_coeffs"]
    r = oracle.recompose(c, shape, B, K, M)
    assert np.abs(r - u).max() <= 1e-12 * np.abs(u).max()


def test_zero_fill_outside_domain():
    """A block that straddles the domain edge sees zeros beyond it (Sec. III-D):
    the ragged field's coefficients equal those of the field padded with 0."""
    u = fields.gaussian_bumps((11, 13, 10), seed=3).astype(np.float64)
    pad = np.zeros((18, 18, 18))
    pad[:11, :13, :10] = u
    cu = oracle.decompose(u, 9, 2, 0)
    cp = oracle.decompose(pad, 9, 2, 0)
    np.testing.assert_array_equal(cu, cp)


def test_block_coeffs_match_full_decomposition():
    u = fields.gaussian_bumps((20, 23, 17), seed=5).astype(np.float64)
    B, K = 9, 2
    p = oracle.plan(u.shape, B, K, 0)
    full = oracle.decompose(u, B, K, 0)
    for b in [0, 5, p["nblocks"] - 1]:
        c, _ = oracle.block_coeffs(u, B, K, b)
        np.testing.assert_array_equal(c, full[b * p["per_block"]:(b + 1) * p["per_block"]])
