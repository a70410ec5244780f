"""The floating-point round-off margin of the L-inf guarantee, measured.

The quantiser's budget is tau' = tau - kappa eps (N+1) max|u| with kappa = 8
(eps = 2^-24 for FP32 fields, 2^-53 for FP64).  The margin has to cover the
round-off of the recomposition done in the field's precision.  Measured here,
without quantisation, on the three single-field workloads (65^3 bumps FP32
B9K3M0, 513^3 k^-5/3 GRF FP32 B17K2M2, 385x385x257 fronts-and-tubes FP64
B9K2M2):
  * recompose error: the GPU's recomposition of the GPU's coefficients, in the
    field's precision, against the oracle's FP64 recomposition of the same
    coefficients;
  * round trip: recompose(decompose(u)) on the GPU against u.
Each is expressed as kappa_eff = error / (eps (N+1) max|u|); the margin keeps
kappa >= 2 kappa_eff."""
import numpy as np
import pytest
import torch

import fields
import oracle

from _util import record

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KAPPA = 8.0

CASES = [
    ("bumps65_f32_b9k3m0", (65, 65, 65), np.float32, 9, 3, 0),
    ("grf513_f32_b17k2m2", (513, 513, 513), np.float32, 17, 2, 2),
    ("roi385_f64_b9k2m2", (385, 385, 257), np.float64, 9, 2, 2),
]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


def _field(name, shape):
    if name.startswith("bumps"):
        return torch.from_numpy(fields.gaussian_bumps(shape, seed=1)).to(DEV)
    if name.startswith("grf"):
        return fields.power_law_grf(shape, seed=2, dtype=torch.float32, device=DEV).contiguous()
    return fields.roi_field(shape, seed=3, device=DEV).contiguous()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_roundoff_margin(bm, case):
    name, shape, dt, B, K, M = case
    t = _field(name, shape)
    assert t.dtype == (torch.float64 if dt == np.float64 else torch.float32)
    eps = 2.0 ** -53 if dt == np.float64 else 2.0 ** -24
    N = K + M
    maxabs = float(t.abs().max())
    unit = eps * (N + 1) * maxabs
    c = bm.decompose(t, block=B, levels=K, global_levels=M)
    r = bm.recompose(c, shape, block=B, levels=K, global_levels=M)
    trip = float((r.double() - t.double()).abs().max())
    exact = oracle.recompose(c.double().cpu().numpy(), shape, B, K, M)
    rec = float(np.abs(r.double().cpu().numpy() - exact).max())
    record(test="roundoff_margin", label=name, kappa=KAPPA, kappa_eff_recompose=rec / unit,
           kappa_eff_round_trip=trip / unit, max_abs=maxabs)
    assert rec / unit <= KAPPA / 2, rec / unit
    assert trip / unit <= KAPPA / 2, trip / unit
