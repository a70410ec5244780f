"""Host-side plan of the CUDA library against the oracle's plan, on the CPU.

`bm_coeff_count` and `bm_compress_bound` run on the host only; the library's
plan (bm_plan.cpp) and the oracle's plan are written independently, so their
coefficient counts must agree for every shape and parameter set, including
ragged shapes, single-block fields, global levels that stop coarsening and
several re-blocking rounds.  Unsupported parameter sets must be refused by
both rather than planned differently.
"""
import itertools

import numpy as np
import pytest

import oracle

SHAPES = [(2, 3, 2), (9, 9, 9), (10, 9, 8), (17, 17, 17), (18, 35, 52), (40, 37, 45), (65, 65, 65),
          (33, 5, 70), (129, 17, 3), (100, 101, 102),
          # 1-D and 2-D fields and explicit extents of 1
          (500,), (3,), (120, 91), (2, 3), (40, 1, 23), (1, 1, 300), (300, 1, 1)]
PARAMS = [(9, k, m) for k in (1, 2, 3) for m in (0, 1, 2, 3)] + [(17, k, m) for k in (1, 2, 3, 4) for m in (0, 1, 2)] \
    + [(8, k, m) for k in (1, 2, 3) for m in (0, 2)] + [(16, k, m) for k in (1, 3) for m in (0, 1)] + [(5, 1, 1), (33, 2, 1)]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    return m


@pytest.mark.parametrize("B,K,M", PARAMS)
def test_coefficient_counts_match_the_oracle(bm, B, K, M):
    for shape in SHAPES:
        try:
            want = oracle.plan(shape, B, K, M)["n_coeffs"]
        except Exception:
            want = None
        try:
            got = bm.coeff_count(shape, B, K, M)
        except Exception:
            got = None
        assert got == want, (shape, B, K, M, got, want)


@pytest.mark.parametrize("R", [2, 3])
def test_coefficient_counts_match_the_oracle_with_rounds(bm, R):
    for shape, (B, K, M) in itertools.product(SHAPES[2:8], [(9, 1, 1), (9, 1, 2), (17, 1, 1), (9, 2, 0), (8, 1, 1),
                                                           (16, 2, 0)]):
        try:
            want = oracle.plan(shape, B, K, M, R)["n_coeffs"]
        except Exception:
            want = None
        try:
            got = bm.coeff_count(shape, B, K, M, rounds=R)
        except Exception:
            got = None
        assert got == want, (shape, B, K, M, R, got, want)


def test_compress_bound_is_the_raw_stream_size(bm):
    import torch

    for shape in SHAPES:
        n = int(np.prod(shape))
        assert bm.compress_bound(shape, torch.float32) == 256 + 4 * n
        assert bm.compress_bound(shape, torch.float64) == 256 + 8 * n
