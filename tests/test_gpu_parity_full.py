"""Parity at the benchmark's own size: the 513^3 FP32 Gaussian random field
(E(k) ~ k^-5/3, seed 2), B = 17, K = 2, M = 2, at the four relative
tolerances 1e-2 .. 1e-5, through the C ABI in the launch configuration the
benchmark times, element by element against the oracle: codes identical
except explained +-1 flips (counted inside and outside the 1e-6 window), the
hard gate (the oracle's quantiser on the GPU's coefficients gives the GPU's
codes exactly), the q table and tiers bit-exact, and the L-inf bound at every
node."""
import numpy as np
import pytest
import torch

import fields
import oracle

from _util import coef_tol, flip_counts, hard_gate, q_per_coeff, record

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPE = (513, 513, 513)
B, K, M = 17, 2, 2


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


@pytest.fixture(scope="module")
def grf513(bm):
    t = fields.power_law_grf(SHAPE, seed=2, dtype=torch.float32, device=DEV).contiguous()
    u = t.cpu().numpy()
    coef_gpu = bm.decompose(t, block=B, levels=K, global_levels=M).cpu().numpy()
    coef_ora = oracle.decompose(u.astype(np.float64), B, K, M)
    err = float(np.abs(coef_gpu.astype(np.float64) - coef_ora).max())
    return t, u, coef_gpu, coef_ora, err


def test_grf513_decompose_matches_oracle(grf513):
    _, u, _, _, err = grf513
    record(test="decompose_full", label="grf513", max_coef_err_over_maxabs=err / float(np.abs(u).max()))
    assert err <= coef_tol(u), err


@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-4, 1e-5])
def test_grf513_compress_parity(bm, grf513, tol):
    t, u, coef_gpu, coef_ora, _ = grf513
    sg = bm.compress(t, tol, mode="rel", block=B, levels=K, global_levels=M).cpu().numpy()
    so, co = oracle.compress(u, tol, rel=True, B=B, K=K, M=M, want_codes=True)
    hg, ho = oracle.stream_header(sg), oracle.stream_header(so)
    assert hg["raw"] == ho["raw"]
    d = bm.decompress(torch.from_numpy(sg).to(DEV))
    maxabs = float(np.abs(u).max())
    err = float((d.double() - t.double()).abs().max())
    assert err <= tol * maxabs
    if hg["raw"]:
        np.testing.assert_array_equal(sg, so)
        record(test="compress_parity_full", label="grf513", tol=tol, raw=True, max_err_over_tau=err / (tol * maxabs))
        return
    for k in ["K", "M", "chunk", "radius", "n_tiers", "m", "nb", "n_symbols", "n_chunks", "max_abs", "margin",
              "off_tiers", "off_qtab", "off_chunks"]:
        assert hg[k] == ho[k], k
    np.testing.assert_array_equal(sg[ho["off_tiers"]:ho["off_chunks"]], so[ho["off_tiers"]:ho["off_chunks"]])
    cg = bm.stream_codes(torch.from_numpy(sg).to(DEV)).cpu().numpy()
    q = q_per_coeff(so)
    fc = flip_counts(cg, co, coef_ora, q, coef_tol(u))
    gate = hard_gate(cg, coef_gpu, q, False)
    record(test="compress_parity_full", label="grf513", shape=list(SHAPE), tol=tol, hard_gate_mismatches=gate,
           max_err_over_tau=err / (tol * maxabs), cr=u.nbytes / sg.size, oracle_cr=u.nbytes / so.size,
           n_outliers=hg["n_outliers"], **fc)
    assert gate == 0, gate
    assert fc["unexplained"] == 0, fc
    if fc["flips"] == 0:
        np.testing.assert_array_equal(sg, so)
