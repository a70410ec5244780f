"""Multi-round re-blocking (Sec. III-C): round r+1 re-blocks the gathered
coarse values of round r into B-node blocks, each new block taking the
strictest tolerance among the blocks whose coarse values it holds, and the
level shares are split over R*K + M + 1 parts.  Pinned by exact round trips,
an independent statement of the propagation rule, and the worst-case L-inf
error of the assembled recomposition with two tolerance tiers."""
import numpy as np
import pytest

import fields
import oracle


@pytest.mark.parametrize("shape,B,K,M,R", [((30, 25, 40), 9, 1, 1, 2), ((40, 19, 27), 9, 1, 0, 3),
                                           ((36, 36, 20), 17, 1, 1, 2), ((20, 20, 20), 9, 2, 1, 2)])
def test_round_trip(shape, B, K, M, R):
    u = np.random.default_rng(sum(shape)).standard_normal(shape)
    c = oracle.decompose(u, B, K, M, R)
    assert c.size == oracle.plan(shape, B, K, M, R)["n_coeffs"]
    np.testing.assert_allclose(oracle.recompose(c, shape, B, K, M, R), u, atol=1e-12)


def test_one_round_is_the_single_round_hierarchy():
    u = np.random.default_rng(3).standard_normal((25, 30, 20))
    np.testing.assert_array_equal(oracle.decompose(u, 9, 2, 1, 1), oracle.decompose(u, 9, 2, 1))
    a = oracle.compress(u, 1e-3, B=9, K=2, M=1, R=1)
    b = oracle.compress(u, 1e-3, B=9, K=2, M=1)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,B,K,R", [((60, 47, 33), 9, 1, 3), ((80, 40, 52), 17, 1, 2), ((50, 50, 50), 9, 2, 2)])
def test_propagation_is_the_minimum_over_contributing_blocks(shape, B, K, R):
    rng = np.random.default_rng(7)
    nb, _ = oracle.rounds(shape, B, K, R)
    t0 = rng.integers(0, 3, size=nb[0]).astype(np.uint8)
    nbs, tiers = oracle.rounds(shape, B, K, R, t0)
    m = B
    for _ in range(K):
        m = m // 2 + 1
    S = np.array(shape)
    for r in range(R - 1):
        nb_r = -(-S // B)
        S_next = nb_r * m
        nb_n = -(-S_next // B)
        prev = tiers[r].reshape(tuple(nb_r))
        want = np.full(tuple(nb_n), 255, dtype=np.uint8)
        # every in-domain node of the next round's grid belongs to the round-r block index // m
        for j0 in range(nb_n[0]):
            for j1 in range(nb_n[1]):
                for j2 in range(nb_n[2]):
                    idx = [np.arange(j * B, min((j + 1) * B, S_next[d])) // m for d, j in enumerate((j0, j1, j2))]
                    owners = prev[np.ix_(np.unique(idx[0]), np.unique(idx[1]), np.unique(idx[2]))]
                    want[j0, j1, j2] = owners.min()
        np.testing.assert_array_equal(tiers[r + 1].reshape(tuple(nb_n)), want)
        S = S_next


def _q_per_coeff_rounds(shape, B, K, M, R, q, ntiers, tiers):
    counts, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        counts.append(n ** 3 - c ** 3)
        n = c
    p = oracle.plan(shape, B, K, M, R)
    parts = []
    for r in range(R):
        for t in tiers[r]:
            parts += [np.full(c, q[int(t) * K + l]) for l, c in enumerate(counts)]
    parts += [np.full(c, q[ntiers * K + l]) for l, c in enumerate(p["global_counts"])]
    parts.append(np.full(p["coarsest"], q[ntiers * K + M]))
    return np.concatenate(parts), p


@pytest.mark.parametrize("shape,B,K,M,R", [((18, 18, 9), 9, 1, 1, 2), ((27, 9, 9), 9, 1, 0, 2)])
def test_linf_bound_with_tiers_across_rounds(shape, B, K, M, R):
    p = oracle.plan(shape, B, K, M, R)
    nc = p["n_coeffs"]
    A = np.zeros((int(np.prod(shape)), nc))
    e = np.zeros(nc)
    for j in range(nc):
        e[j] = 1.0
        A[:, j] = oracle.recompose(e, shape, B, K, M, R).ravel()
        e[j] = 0.0
    nb, _ = oracle.rounds(shape, B, K, R)
    t0 = np.ones(nb[0], dtype=np.uint8)
    t0[0] = 0  # the first block is the strict region
    _, tiers = oracle.rounds(shape, B, K, R, t0)
    taus = [0.1, 1.0]
    q, margin, raw = oracle.budget(shape, B, K, M, taus, 0.0, True, R)
    assert margin == 0.0 and not raw
    qc, _ = _q_per_coeff_rounds(shape, B, K, M, R, q, 2, tiers)
    worst = (np.abs(A) @ (qc / 2.0)).reshape(shape)
    tau_node = np.full(shape, 1.0)
    tau_node[:B, :B, :B] = 0.1
    assert np.all(worst <= tau_node * (1 + 1e-12))
    # without propagation the strict block's bound would fail: its coarse values
    # are re-blocked with the loose neighbours
    tiers_np = [tiers[0]] + [np.ones_like(t) for t in tiers[1:]]
    qc2, _ = _q_per_coeff_rounds(shape, B, K, M, R, q, 2, tiers_np)
    worst2 = (np.abs(A) @ (qc2 / 2.0)).reshape(shape)
    assert (worst2 > tau_node * (1 + 1e-12)).any()


def test_roi_bound_end_to_end_with_rounds():
    u = fields.roi_field((40, 37, 29), seed=4).numpy()
    B, K, M, R = 9, 1, 1, 2
    roi_mask = fields.gradient_roi(u, B)
    roi = np.where(roi_mask, 1e-5, 1e-2)
    s = oracle.compress(u, 1e-2, rel=True, roi=roi, B=B, K=K, M=M, R=R)
    assert oracle.stream_header(s)["R"] == R
    d = oracle.decompress(s)
    mx = np.abs(u).max()
    tau_node = np.repeat(np.repeat(np.repeat(roi, B, 0), B, 1), B, 2)[: u.shape[0], : u.shape[1], : u.shape[2]] * mx
    assert np.all(np.abs(d - u) <= tau_node)
