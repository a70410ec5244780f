"""Multi-round re-blocking (Sec. III-C) through the C ABI against the oracle:
coefficients, recomposition, tolerance propagation (the stream's block-tier
section bit-exact), codes with explained flips only, the L-inf bound per
region, byte-identical streams when the codes agree, and the GPU decoding the
oracle's streams."""
import numpy as np
import pytest
import torch

import fields
import oracle

from _util import flip_counts, hard_gate, per_block_tau, record

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (name, shape, dtype, B, K, M, R)
CASES = [
    ("grf_b9k1m1r2", (40, 37, 45), np.float32, 9, 1, 1, 2),
    ("grf_b9k1m0r3", (52, 35, 70), np.float32, 9, 1, 0, 3),
    ("grf_b17k1m1r2", (70, 61, 53), np.float32, 17, 1, 1, 2),
    ("roi_f64_b9k2m1r2", (47, 41, 33), np.float64, 9, 2, 1, 2),
    # the paper's schedule: 8-node blocks, one level per round, three rounds
    ("grf_b8k1m1r3", (60, 45, 52), np.float32, 8, 1, 1, 3),
    ("roi_f64_b8k1m0r3", (47, 41, 33), np.float64, 8, 1, 0, 3),
]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


def _field(name, shape, dtype):
    u = fields.roi_field(shape, seed=3).numpy() if name.startswith("roi") else fields.power_law_grf(shape, seed=2).numpy()
    return np.ascontiguousarray(u.astype(dtype))


def _coef_tol(u):
    return (1e-5 if u.dtype == np.float32 else 1e-12) * float(np.abs(u).max())


def _q_per_coeff(stream, shape, B, K, M, R):
    h = oracle.stream_header(stream)
    nt = h["n_tiers"]
    nq = nt * K + M + 1
    q = np.asarray(stream[h["off_qtab"]:h["off_qtab"] + 8 * nq]).view(np.float64)
    nbs = oracle.plan_rounds_count(shape, B, K, R)
    if nt > 1:
        flat = np.asarray(stream[h["off_blocktier"]:h["off_blocktier"] + sum(nbs)]).astype(np.int64)
    else:
        flat = np.zeros(sum(nbs), dtype=np.int64)
    counts, n = [], B
    for _ in range(K):
        c = n // 2 + 1
        counts.append(n ** 3 - c ** 3)
        n = c
    per_level = np.concatenate([np.full(c, l) for l, c in enumerate(counts)])
    p = oracle.plan(shape, B, K, M, R)
    parts = [q[(flat[:, None] * K + per_level[None, :]).ravel()]]
    for l, c in enumerate(p["global_counts"]):
        parts.append(np.full(c, q[nt * K + l]))
    parts.append(np.full(p["coarsest"], q[nt * K + M]))
    return np.concatenate(parts)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_decompose_recompose_match_oracle(bm, case):
    name, shape, dt, B, K, M, R = case
    u = _field(name, shape, dt)
    t = torch.from_numpy(u).to(DEV)
    cg = bm.decompose(t, B, K, M, rounds=R).double().cpu().numpy()
    co = oracle.decompose(u.astype(np.float64), B, K, M, R)
    assert cg.shape == co.shape
    np.testing.assert_allclose(cg, co, atol=_coef_tol(u))
    rg = bm.recompose(torch.from_numpy(co.astype(dt)).to(DEV), shape, B, K, M, rounds=R).double().cpu().numpy()
    ro = oracle.recompose(co.astype(dt).astype(np.float64), shape, B, K, M, R)
    np.testing.assert_allclose(rg, ro, atol=10 * _coef_tol(u))


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_compress_parity_with_rounds(bm, case, tol):
    name, shape, dt, B, K, M, R = case
    u = _field(name, shape, dt)
    roi = None
    if name.startswith("roi"):
        roi = np.where(fields.gradient_roi(u, B), tol * 1e-2, tol)
    sg = bm.compress(torch.from_numpy(u).to(DEV), tol, mode="rel", roi=roi, block=B, levels=K, global_levels=M,
                     rounds=R).cpu().numpy()
    so, co = oracle.compress(u, tol, rel=True, roi=roi, B=B, K=K, M=M, R=R, want_codes=True)
    hg, ho = oracle.stream_header(sg), oracle.stream_header(so)
    assert hg["raw"] == ho["raw"]
    d = bm.decompress(torch.from_numpy(sg).to(DEV)).cpu().numpy().astype(np.float64)
    tau = per_block_tau(sg, shape, B) if not hg["raw"] else 0.0
    assert np.all(np.abs(d - u) <= tau)
    if hg["raw"]:
        np.testing.assert_array_equal(sg, so)
        return
    assert hg["R"] == ho["R"] == R
    for k in ["K", "M", "n_tiers", "n_symbols", "n_chunks", "max_abs", "margin", "off_qtab", "off_blocktier",
              "off_chunks"]:
        assert hg[k] == ho[k], k
    # tiers, q table and every round's propagated block tiers bit-exact
    np.testing.assert_array_equal(sg[ho["off_tiers"]:ho["off_chunks"]], so[ho["off_tiers"]:ho["off_chunks"]])
    cg = bm.stream_codes(torch.from_numpy(sg).to(DEV)).cpu().numpy()
    coef = oracle.decompose(u.astype(np.float64), B, K, M, R)
    q = _q_per_coeff(so, shape, B, K, M, R)
    fc = flip_counts(cg, co, coef, q, _coef_tol(u))
    cgpu = bm.decompose(torch.from_numpy(u).to(DEV), B, K, M, rounds=R).cpu().numpy()
    gate = hard_gate(cg, cgpu, q, dt == np.float64)
    record(test="compress_parity_rounds", label=name, shape=list(shape), dtype=str(u.dtype), B=B, K=K, M=M, R=R,
           tol=tol, hard_gate_mismatches=gate, **fc)
    assert gate == 0, gate
    assert fc["unexplained"] == 0, fc
    if fc["flips"] == 0:
        np.testing.assert_array_equal(sg, so)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gpu_decodes_oracle_stream_with_rounds(bm, case):
    name, shape, dt, B, K, M, R = case
    u = _field(name, shape, dt)
    so = oracle.compress(u, 1e-3, rel=True, B=B, K=K, M=M, R=R)
    do = oracle.decompress(so).astype(np.float64)
    dg = bm.decompress(torch.from_numpy(so).to(DEV)).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(dg, do, atol=10 * _coef_tol(u))
