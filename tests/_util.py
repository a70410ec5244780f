"""Helpers shared by the GPU parity tests (no method arithmetic here: they only
index streams and compare arrays)."""
import numpy as np

import oracle


def local_counts(B, K):
    out, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        out.append(n ** 3 - c ** 3)
        n = c
    return out


def q_per_coeff(stream):
    """Quantiser width of every coefficient, read from a stream's q table and
    block tiers (stream order)."""
    h = oracle.stream_header(stream)
    B, K, M, nt = h["B"], h["K"], h["M"], h["n_tiers"]
    p = oracle.plan(h["shape"], B, K, M)
    nq = nt * K + M + 1
    q = np.asarray(stream[h["off_qtab"]:h["off_qtab"] + 8 * nq]).view(np.float64)
    if nt > 1:
        tier = np.asarray(stream[h["off_blocktier"]:h["off_blocktier"] + p["nblocks"]]).astype(np.int64)
    else:
        tier = np.zeros(p["nblocks"], dtype=np.int64)
    lc = local_counts(B, K)
    per_level = np.concatenate([np.full(c, l) for l, c in enumerate(lc)]) if K else np.zeros(0, np.int64)
    local = q[(tier[:, None] * K + per_level[None, :]).ravel()]
    parts = [local]
    for l, c in enumerate(p["global_counts"]):
        parts.append(np.full(c, q[nt * K + l]))
    parts.append(np.full(p["coarsest"], q[nt * K + M]))
    return np.concatenate(parts)


def classify_flips(codes_gpu, codes_ora, coef_ora, q, coef_tol):
    """Codes may differ by one bin where the oracle's coefficient lies within
    the coefficient tolerance of the edge between the two bins.  Returns
    (n_flips, n_flips_within_1e-6_relative, n_unexplained)."""
    g = np.asarray(codes_gpu, dtype=np.int64)
    o = np.asarray(codes_ora, dtype=np.int64)
    diff = np.flatnonzero(g != o)
    if diff.size == 0:
        return 0, 0, 0
    step = np.abs(g[diff] - o[diff])
    lo = np.minimum(g[diff], o[diff])
    edge = (lo + 0.5) * q[diff]
    dist = np.abs(coef_ora[diff] - edge)
    explained = (step == 1) & (dist <= coef_tol + 4 * np.finfo(np.float32).eps * np.abs(edge))
    within = (step == 1) & (dist <= 1e-6 * np.maximum(np.abs(coef_ora[diff]), q[diff]))
    return int(diff.size), int(within.sum()), int((~explained).sum())


def per_block_tau(stream, shape, B):
    """Absolute tolerance of every node, from the stream's tiers and block tiers."""
    h = oracle.stream_header(stream)
    nt = h["n_tiers"]
    tiers = np.asarray(stream[h["off_tiers"]:h["off_tiers"] + 8 * nt]).view(np.float64)
    nb = h["nb"]
    if nt > 1:
        tier = np.asarray(stream[h["off_blocktier"]:h["off_blocktier"] + int(np.prod(nb))]).astype(np.int64)
    else:
        tier = np.zeros(int(np.prod(nb)), dtype=np.int64)
    t = tiers[tier].reshape(nb)
    t = np.repeat(np.repeat(np.repeat(t, B, 0), B, 1), B, 2)
    return t[: shape[0], : shape[1], : shape[2]]
