"""Helpers shared by the GPU parity tests (no method arithmetic here: they only
index streams and compare arrays)."""
import numpy as np

import oracle


def block_edges(shape3, B):
    """Block edge per dimension of a 3-D shape: B, or 1 along an extent of 1."""
    return [1 if n == 1 else B for n in shape3]


def local_counts(B, K, shape3=(2, 2, 2)):
    """Coefficients of each in-cache level inside one block (a dimension of
    extent 1 is neither blocked nor coarsened)."""
    out, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        nn = cc = 1
        for e in shape3:
            nn *= 1 if e == 1 else n
            cc *= 1 if e == 1 else c
        out.append(nn - cc)
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
    lc = local_counts(B, K, h["shape"])
    per_level = np.concatenate([np.full(c, l) for l, c in enumerate(lc)]) if K else np.zeros(0, np.int64)
    local = q[(tier[:, None] * K + per_level[None, :]).ravel()]
    parts = [local]
    for l, c in enumerate(p["global_counts"]):
        parts.append(np.full(c, q[nt * K + l]))
    parts.append(np.full(p["coarsest"], q[nt * K + M]))
    return np.concatenate(parts)


# Parity figures of the GPU tests (flip counts, hard-gate mismatches, errors),
# printed at the end of the session and written to $BM_PARITY_LOG if set.
PARITY_RECORDS = []


def record(**kw):
    PARITY_RECORDS.append(kw)


def flip_counts(codes_gpu, codes_ora, coef_ora, q, coef_tol):
    """Codes that differ between the GPU and the oracle ("flips"), split by
    where the oracle's coefficient lies: within 1e-6 relative (of max(|c|, q))
    of the edge between the two bins, or outside that window.  A flip is
    explained when it is one bin and the coefficient lies within the
    coefficient tolerance of that edge (the GPU's coefficient, computed in
    the field's precision, may sit on the other side)."""
    g = np.asarray(codes_gpu, dtype=np.int64)
    o = np.asarray(codes_ora, dtype=np.int64)
    diff = np.flatnonzero(g != o)
    if diff.size == 0:
        return {"flips": 0, "within_1e-6": 0, "outside_1e-6": 0, "unexplained": 0, "n": int(g.size)}
    step = np.abs(g[diff] - o[diff])
    lo = np.minimum(g[diff], o[diff])
    edge = (lo + 0.5) * q[diff]
    dist = np.abs(coef_ora[diff] - edge)
    explained = (step == 1) & (dist <= coef_tol + 4 * np.finfo(np.float32).eps * np.abs(edge))
    within = (step == 1) & (dist <= 1e-6 * np.maximum(np.abs(coef_ora[diff]), q[diff]))
    return {"flips": int(diff.size), "within_1e-6": int(within.sum()), "outside_1e-6": int((~within).sum()),
            "unexplained": int((~explained).sum()), "n": int(g.size)}


def classify_flips(codes_gpu, codes_ora, coef_ora, q, coef_tol):
    """(n_flips, n_flips_within_1e-6_relative, n_unexplained) of flip_counts."""
    f = flip_counts(codes_gpu, codes_ora, coef_ora, q, coef_tol)
    return f["flips"], f["within_1e-6"], f["unexplained"]


def hard_gate(codes_gpu, coef_gpu, q, f64):
    """The oracle's quantiser applied to the GPU's own coefficients (its
    full-precision decomposition output) must give the GPU's codes exactly:
    the quantiser, the level/tier widths and the stream order are then
    identical, and every remaining code difference from the oracle comes from
    the coefficients alone.  Returns the number of mismatches."""
    codes, ovf = oracle.quantize_array(np.asarray(coef_gpu, dtype=np.float64), q, f64)
    assert not ovf.any()
    return int(np.count_nonzero(codes != np.asarray(codes_gpu, dtype=np.int64)))


def per_block_tau(stream, shape, B):
    """Absolute tolerance of every node, from the stream's tiers and block
    tiers, in the field's own shape."""
    h = oracle.stream_header(stream)
    nt = h["n_tiers"]
    tiers = np.asarray(stream[h["off_tiers"]:h["off_tiers"] + 8 * nt]).view(np.float64)
    nb = h["nb"]
    if nt > 1:
        tier = np.asarray(stream[h["off_blocktier"]:h["off_blocktier"] + int(np.prod(nb))]).astype(np.int64)
    else:
        tier = np.zeros(int(np.prod(nb)), dtype=np.int64)
    s3 = h["shape"]
    t = tiers[tier].reshape(nb)
    for ax, e in enumerate(block_edges(s3, B)):
        t = np.repeat(t, e, ax)
    return t[: s3[0], : s3[1], : s3[2]].reshape(shape)


def coef_tol(u):
    """Coefficient tolerance of the parity bar: 1e-5 (FP32) or 1e-12 (FP64)
    of max|u|."""
    return (1e-5 if u.dtype == np.float32 else 1e-12) * float(np.abs(u).max())


def check_stream_parity(bm, u, sg, tol, mode, B, K, M, roi=None, label="", dev="cuda:0", radius=32768):
    """A GPU stream sg of field u against the oracle's stream of the same
    field and arguments: raw decision, the L-inf bound at every node of every
    region (GPU decode), header fields and the tier / q tables bit-exact,
    codes identical except explained +-1 flips (counted inside and outside
    the 1e-6 window and recorded), the hard gate, and the whole stream
    byte-identical when no code flips.  Returns the oracle's codes (None for
    a raw stream)."""
    import torch

    shape = u.shape
    f64 = u.dtype == np.float64
    so, co = oracle.compress(u, tol, rel=(mode == "rel"), roi=roi, B=B, K=K, M=M, radius=radius, want_codes=True)
    hg, ho = oracle.stream_header(sg), oracle.stream_header(so)
    assert hg["raw"] == ho["raw"]
    d = bm.decompress(torch.from_numpy(sg).to(dev)).cpu().numpy().astype(np.float64)
    tau = per_block_tau(sg, shape, B) if not hg["raw"] else 0.0
    err = np.abs(d - u.astype(np.float64))
    assert np.all(err <= tau)
    if hg["raw"]:
        np.testing.assert_array_equal(sg, so)
        record(test="compress_parity", label=label, shape=list(shape), dtype=str(u.dtype), B=B, K=K, M=M, tol=tol,
               mode=mode, raw=True)
        return None
    for k in ["K", "M", "chunk", "radius", "n_tiers", "m", "nb", "n_symbols", "n_chunks", "max_abs", "margin",
              "off_tiers", "off_qtab", "off_blocktier", "off_chunks"]:
        assert hg[k] == ho[k], k
    a, b = ho["off_tiers"], ho["off_chunks"]
    np.testing.assert_array_equal(sg[a:b], so[a:b])
    cg = bm.stream_codes(torch.from_numpy(sg).to(dev)).cpu().numpy()
    coef = oracle.decompose(u.astype(np.float64), B, K, M)
    q = q_per_coeff(so)
    fc = flip_counts(cg, co, coef, q, coef_tol(u))
    cgpu = bm.decompose(torch.from_numpy(u).to(dev), block=B, levels=K, global_levels=M).cpu().numpy()
    gate = hard_gate(cg, cgpu, q, f64)
    worst = float((err / np.maximum(tau, np.finfo(np.float64).tiny)).max())
    record(test="compress_parity", label=label, shape=list(shape), dtype=str(u.dtype), B=B, K=K, M=M, tol=tol,
           mode=mode, radius=radius, n_tiers=ho["n_tiers"], n_outliers=ho["n_outliers"],
           hard_gate_mismatches=gate, max_err_over_tau=worst,
           cr=float(u.nbytes) / sg.size, **fc)
    assert gate == 0, gate
    assert fc["unexplained"] == 0, fc
    if fc["flips"] == 0:
        np.testing.assert_array_equal(sg, so)  # whole stream bit-exact
    if f64:
        assert fc["flips"] <= 2
    return np.asarray(co)
