"""Alg. 1 parameter selection and the Eq. 1 model on the host (no GPU): the
selection is the feasible (K, M) pair largest in (M, -K), the knee follows the
closed form of Eq. 1, predictions grow with the field."""
import pytest

import paper_2609_00205_gb300 as bm


@pytest.fixture(scope="module")
def model():
    import __graft_entry__

    __graft_entry__.build()
    bm.load()
    m = bm.PerfModel()
    m.block_latency_ms = 0.02
    m.block_peak_per_ms = 60000.0
    m.global_ms = 0.01
    m.global_ms_per_node = 2e-8
    m.hist_ms = 0.01
    m.hist_ms_per_symbol = 1e-9
    m.codebook_ms = 0.1
    m.encode_ms = 0.01
    m.encode_ms_per_symbol = 2.5e-9
    m.other_ms = 0.15
    m.block_nodes = 17
    m.incache_levels = 2
    m.dtype = bm.BM_F32
    return m


def test_knee_closed_form(model):
    n0 = model.block_peak_per_ms * model.block_latency_ms
    for f in (0.5, 0.9, 0.99):
        n = bm.perf_model_knee(model, f)
        # Eq. 1 at that block count reaches the fraction of the peak
        tp = n / (model.block_latency_ms + n / model.block_peak_per_ms)
        assert abs(tp / model.block_peak_per_ms - f) < 1e-12
        assert abs(n - n0 * f / (1 - f)) < 1e-9 * n


def test_prediction_grows_with_the_field(model):
    a = bm.predict_ms(model, (129, 129, 129))
    b = bm.predict_ms(model, (257, 257, 257))
    c = bm.predict_ms(model, (513, 513, 513))
    assert 0 < a < b < c


def test_selection_is_alg1(model):
    shape = (257, 257, 257)
    # generous budget: the most global levels, then the fewest in-cache levels
    p, t = bm.select_params(model, shape, 1e9)
    feasible = []
    for K in range(1, 5):
        # candidates: global levels while some dimension of the gathered grid still coarsens
        m = 17
        for _ in range(K):
            m = m // 2 + 1
        g = [((n + 16) // 17) * m for n in shape]
        mmax = 0
        while mmax < 16 and max(g) > 2:
            g = [v // 2 + 1 if v > 2 else v for v in g]
            mmax += 1
        for M in range(0, mmax + 1):
            feasible.append((M, -K, bm.predict_ms(model, shape, 17, K, M if M else -1)))
    best = max(feasible, key=lambda z: (z[0], z[1]))
    assert (p["global_levels"], -p["levels"]) == (best[0], best[1])
    # a budget between two candidates' predictions excludes the slower ones
    times = sorted(set(round(z[2], 9) for z in feasible))
    mid = (times[0] + times[1]) / 2
    p2, t2 = bm.select_params(model, shape, mid)
    assert t2 <= mid
    ok = [z for z in feasible if z[2] <= mid]
    best2 = max(ok, key=lambda z: (z[0], z[1]))
    assert (p2["global_levels"], -p2["levels"]) == (best2[0], best2[1])
    with pytest.raises(bm.BlockMGARDError):
        bm.select_params(model, shape, times[0] / 2)
