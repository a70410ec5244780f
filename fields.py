"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module draws random fields, ROI masks and symbol sequences only; it holds
none of the compressor's arithmetic (no interpolation, mass matrices,
quantisation or entropy coding), so both the CUDA path and the CPU oracle can
consume its outputs without sharing any method code.

The fields stand in for the SDRBench datasets the paper evaluates on (NYX,
Hurricane ISABEL, SCALE-LETKF, Miranda, S3D; Table I), which are not available
here.  Shapes, dtypes and value structure follow the workloads below:

* ``gaussian_bumps``   65^3 FP32: sum of 8 Gaussian bumps + N(0, 1e-3) noise.
* ``power_law_grf``    Gaussian random field whose shell-integrated power
                       spectrum is E(k) ~ k^p (p = -5/3, the Kolmogorov
                       spectrum, for the 513^3 FP32 hybrid workload; p = -3 for
                       the ROI background), i.e. |u_hat(k)|^2 ~ k^(p-2) in 3-D;
                       unit variance.
* ``roi_field``        385x385x257 FP64: k^-3 GRF + 12 tanh fronts + 6 vortex tubes.
* ``gradient_roi``     per-block ROI: blocks whose max |grad u| exceeds the 95th
                       percentile of the pointwise |grad u|.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed))


def gaussian_bumps(shape=(65, 65, 65), seed: int = 1, n_bumps: int = 8,
                   noise: float = 1e-3) -> np.ndarray:
    """Sum of ``n_bumps`` Gaussian bumps (centres U[0, n-1]^3, amplitudes
    U[0.5, 2], widths U[4, 12] cells) plus N(0, noise) white noise, FP32."""
    rng = _rng(seed)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    u = np.zeros(shape, dtype=np.float64)
    for _ in range(n_bumps):
        centre = [rng.uniform(0, n - 1) for n in shape]
        amp = rng.uniform(0.5, 2.0)
        width = rng.uniform(4.0, 12.0)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        u += amp * np.exp(-r2 / (2.0 * width * width))
    u += rng.normal(0.0, noise, size=shape)
    return u.astype(np.float32)


def _wavenumber_amplitude(shape, exponent, device):
    """|k|^(exponent/2) on the rfft grid (k in integer-index units), 0 at k=0;
    ``exponent`` is that of the modal spectrum |u_hat(k)|^2."""
    ks = []
    for d, n in enumerate(shape):
        if d == len(shape) - 1:
            k = torch.fft.rfftfreq(n, d=1.0 / n, device=device, dtype=torch.float64)
        else:
            k = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64)
        view = [1] * len(shape)
        view[d] = -1
        ks.append(k.view(view))
    k2 = ks[0] ** 2
    for k in ks[1:]:
        k2 = k2 + k ** 2
    kk = torch.sqrt(k2)
    amp = torch.where(kk > 0, kk.clamp_min(1e-30) ** (exponent / 2.0), torch.zeros_like(kk))
    return amp


def power_law_grf(shape, exponent: float = -5.0 / 3.0, seed: int = 2,
                  dtype=torch.float32, device="cpu") -> torch.Tensor:
    """Gaussian random field whose shell-integrated spectrum is
    E(k) ~ k^exponent, i.e. modal spectrum |u_hat(k)|^2 ~ k^(exponent - (d-1))
    (k = 0 removed), FFT synthesis from seeded white noise, unit variance.

    White noise is drawn on the CPU with a seeded torch generator so every
    device receives the same noise; the FFT runs on ``device``.
    """
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    work = torch.float64 if dtype == torch.float64 else torch.float32
    noise = torch.randn(tuple(shape), generator=gen, dtype=work).to(device)
    spec = torch.fft.rfftn(noise)
    del noise
    amp = _wavenumber_amplitude(shape, exponent - (len(shape) - 1), device).to(spec.real.dtype)
    spec.mul_(amp)
    del amp
    u = torch.fft.irfftn(spec, s=tuple(shape))
    del spec
    u = u - u.mean()
    u = u / u.std()
    return u.to(dtype)


def roi_field(shape=(385, 385, 257), seed: int = 3, device="cpu") -> torch.Tensor:
    """FP64 field: smooth k^-3 GRF background (unit variance) + 12 seeded tanh
    fronts A*tanh((n.x - d)/2) (thickness 2 cells, n uniform on the sphere,
    d inside the domain, A ~ U[0.5, 2]) + 6 Gaussian vortex tubes
    A*exp(-r^2 / (2 s^2)) around random lines (s ~ U[2, 6], A ~ U[0.5, 2])."""
    rng = _rng(seed)
    u = power_law_grf(shape, exponent=-3.0, seed=seed * 1000 + 7,
                      dtype=torch.float64, device=device)
    axes = [torch.arange(n, dtype=torch.float64, device=device) for n in shape]
    X = [a.view([-1 if i == d else 1 for i in range(3)]) for d, a in enumerate(axes)]
    centre_box = np.array(shape, dtype=np.float64) - 1.0
    for _ in range(12):
        nvec = rng.normal(size=3)
        nvec /= np.linalg.norm(nvec)
        p = rng.uniform(0, 1, size=3) * centre_box
        d = float(nvec @ p)
        amp = rng.uniform(0.5, 2.0)
        s = X[0] * nvec[0] + X[1] * nvec[1] + X[2] * nvec[2] - d
        u += amp * torch.tanh(s / 2.0)
    for _ in range(6):
        p = rng.uniform(0, 1, size=3) * centre_box
        t = rng.normal(size=3)
        t /= np.linalg.norm(t)
        sigma = rng.uniform(2.0, 6.0)
        amp = rng.uniform(0.5, 2.0)
        dx = [X[i] - p[i] for i in range(3)]
        along = dx[0] * t[0] + dx[1] * t[1] + dx[2] * t[2]
        r2 = dx[0] ** 2 + dx[1] ** 2 + dx[2] ** 2 - along ** 2
        u += amp * torch.exp(-r2.clamp_min(0.0) / (2.0 * sigma * sigma))
    return u


def gradient_roi(u: np.ndarray, block: int, percentile: float = 95.0) -> np.ndarray:
    """Boolean ROI per block of ``block`` nodes per dim (row-major block grid):
    True where the block's max |grad u| (central differences, one-sided at the
    edges) exceeds the given percentile of the pointwise |grad u|."""
    u64 = np.asarray(u, dtype=np.float64)
    g = np.gradient(u64)
    mag = np.sqrt(sum(gi * gi for gi in g))
    thr = np.percentile(mag, percentile)
    nb = [int(math.ceil(n / block)) for n in u64.shape]
    pad = [(0, nb[d] * block - u64.shape[d]) for d in range(3)]
    magp = np.pad(mag, pad, constant_values=-np.inf)
    blk = magp.reshape(nb[0], block, nb[1], block, nb[2], block).max(axis=(1, 3, 5))
    return blk > thr


def random_roi(nblocks, fraction: float, seed: int) -> np.ndarray:
    """Boolean mask over ``nblocks`` blocks with ``fraction`` of them set."""
    rng = _rng(seed)
    n = int(np.prod(nblocks))
    k = int(round(fraction * n))
    mask = np.zeros(n, dtype=bool)
    mask[rng.choice(n, size=k, replace=False)] = True
    return mask.reshape(nblocks)


def laplace_symbols(n: int, radius: int, scale: float, seed: int,
                    escape_rate: float = 0.0) -> np.ndarray:
    """uint16 symbols code + radius with code ~ round(Laplace(0, scale)),
    clipped to the dictionary; a fraction ``escape_rate`` replaced by 0."""
    rng = _rng(seed)
    code = np.rint(rng.laplace(0.0, scale, size=n)).astype(np.int64)
    code = np.clip(code, -(radius - 1), radius - 1)
    sym = (code + radius).astype(np.uint16)
    if escape_rate > 0:
        sym[rng.random(n) < escape_rate] = 0
    return sym


def smooth_multilinear(shape, coeffs=(0.3, -1.2, 0.7, 2.0, 0.5, -0.25, 0.125, 1.5)) -> np.ndarray:
    """a + b x + c y + d z + e xy + f xz + g yz + h xyz on integer coordinates (FP64)."""
    x, y, z = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    a, b, c, d, e, f, g, h = coeffs
    return a + b * x + c * y + d * z + e * x * y + f * x * z + g * y * z + h * x * y * z
