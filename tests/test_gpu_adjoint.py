"""Adjoint kernels (transposed decomposition / recomposition) through the C ABI.

Checked against the oracle's explicit transpose on small ragged grids, by the
dot-product identity on larger ones, by torch.autograd.gradcheck (FP64, finite
differences) and by central differences of a smoothing loss at 1e-6 relative.
"""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    m.load()
    return m


@pytest.mark.parametrize("shape,B,K,M", [((17, 17, 17), 17, 2, 1), ((20, 19, 22), 9, 2, 1), ((12, 9, 10), 9, 1, 2)])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
def test_adjoints_match_oracle_transpose(bm, shape, B, K, M, dtype, tol):
    rng = np.random.default_rng(sum(shape) + B)
    nc = oracle.plan(shape, B, K, M)["n_coeffs"]
    gcoef = rng.standard_normal(nc)
    gfield = rng.standard_normal(shape)
    want_u = oracle.decompose_adjoint(gcoef, shape, B, K, M)
    want_c = oracle.recompose_adjoint(gfield, shape, B, K, M)
    got_u = bm.decompose_adjoint(torch.tensor(gcoef, dtype=dtype, device=DEV), shape, B, K, M).double().cpu().numpy()
    got_c = bm.recompose_adjoint(torch.tensor(gfield, dtype=dtype, device=DEV), B, K, M).double().cpu().numpy()
    np.testing.assert_allclose(got_u, want_u, atol=tol * np.abs(want_u).max())
    np.testing.assert_allclose(got_c, want_c, atol=tol * np.abs(want_c).max())


@pytest.mark.parametrize("shape,B,K,M", [((33, 33, 33), 17, 2, 2), ((65, 40, 50), 9, 2, 2), ((70, 61, 53), 17, 3, 1)])
def test_dot_product_identity(bm, shape, B, K, M):
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn(shape, generator=g, dtype=torch.float64).to(DEV)
    nc = bm.coeff_count(shape, B, K, M)
    y = torch.randn(nc, generator=g, dtype=torch.float64).to(DEV)
    lhs = torch.dot(bm.decompose(x, B, K, M), y).item()
    rhs = torch.dot(x.ravel(), bm.decompose_adjoint(y, shape, B, K, M).ravel()).item()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    c = torch.randn(nc, generator=g, dtype=torch.float64).to(DEV)
    lhs = torch.dot(bm.recompose(c, shape, B, K, M).ravel(), x.ravel()).item()
    rhs = torch.dot(c, bm.recompose_adjoint(x, B, K, M)).item()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("shape", [(17, 17, 17), (33, 33, 33)])
def test_gradcheck(bm, shape):
    g = torch.Generator(device="cpu").manual_seed(3)
    u = torch.randn(shape, generator=g, dtype=torch.float64).to(DEV).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: bm.decompose_ad(t, 17, 2, 2), (u,), fast_mode=True)
    nc = bm.coeff_count(shape, 17, 2, 2)
    c = torch.randn(nc, generator=g, dtype=torch.float64).to(DEV).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: bm.recompose_ad(t, shape, 17, 2, 2), (c,), fast_mode=True)


def _loss(bm, c, shape, target):
    u = bm.recompose_ad(c, shape, 17, 2, 2)
    gx = [torch.diff(u, dim=d) for d in range(3)]
    return ((u - target) ** 2).sum() + 0.1 * sum((t ** 2).sum() for t in gx)


def test_loss_gradient_central_differences(bm):
    shape = (33, 33, 33)
    u0 = fields.power_law_grf(shape, seed=5, dtype=torch.float64, device=DEV)
    c = bm.decompose(u0.contiguous(), 17, 2, 2).clone().requires_grad_(True)
    g = torch.Generator(device="cpu").manual_seed(11)
    target = u0 + 0.1 * torch.randn(shape, generator=g, dtype=torch.float64).to(DEV)
    loss = _loss(bm, c, shape, target)
    (grad,) = torch.autograd.grad(loss, c)
    d = torch.randn(c.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-4
    with torch.no_grad():
        fd = (_loss(bm, c + eps * d, shape, target) - _loss(bm, c - eps * d, shape, target)) / (2 * eps)
    ad = torch.dot(grad, d)
    # the loss is quadratic in c: central differences are exact up to rounding
    assert abs(fd.item() - ad.item()) <= 1e-6 * abs(ad.item())
