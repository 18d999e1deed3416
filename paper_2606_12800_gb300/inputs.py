"""Seeded synthetic inputs: fractal DEMs, rainfall fields and tile batches.

This module is shared by the GPU path's tests/benchmark and by the CPU oracle's
tests.  It holds none of the flow-routing arithmetic: it only draws random
surfaces.  They stand in for the depression-filled Copernicus DEM of Colorado
used in the paper's experiments (Sec. 4), which is not available here; unlike
that DEM they are not depression-filled, so interior pits are sinks.

Recipe (spectral fractal surface):
  1. complex Gaussian Fourier modes A(k) = (N(0,1) + i N(0,1)) * |k|^(-beta/2),
     integer wavenumbers k (cycles per domain) on the FFT grid, A(0) = 0;
  2. z = Re(ifft2(A)), min-max scaled to [0, 1000] m;
  3. + planar tilt  t * dx * (nx - 1 - x)  (descends toward +x);
  4. + jitter U[0, 1e-4) m;
  5. rounded once to float32.
Rain is U[0, 1) float32 drawn from ``seed + 1``.

CPU generation uses numpy's PCG64 in FP64 (bit-identical on every machine with
numpy >= 1.17).  Grids too large for host FFTs (>= 16384^2) are drawn on the GPU
with torch in complex64; those surfaces differ from the CPU ones for the same
seed, and every check on them reads back the same float32 bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

Z_RANGE_M = 1000.0
JITTER_M = 1e-4


def fractal_dem(n_y: int, n_x: int, beta: float = 2.0, tilt: float = 0.01,
                seed: int = 0, dx: float = 30.0, jitter: float = JITTER_M) -> np.ndarray:
    """Seeded fractal DEM (float32, shape (n_y, n_x)), numpy FP64 recipe."""
    rng = np.random.default_rng(seed)
    ky = np.fft.fftfreq(n_y) * n_y
    kx = np.fft.fftfreq(n_x) * n_x
    kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    kk[0, 0] = 1.0
    amp = kk ** (-beta / 2.0)
    amp[0, 0] = 0.0
    re = rng.standard_normal((n_y, n_x))
    im = rng.standard_normal((n_y, n_x))
    z = np.fft.ifft2((re + 1j * im) * amp).real
    lo, hi = z.min(), z.max()
    z = (z - lo) / (hi - lo) * Z_RANGE_M if hi > lo else np.zeros_like(z)
    if tilt:
        z = z + tilt * dx * (n_x - 1 - np.arange(n_x, dtype=np.float64))[None, :]
    if jitter:
        z = z + rng.uniform(0.0, jitter, size=(n_y, n_x))
    return z.astype(np.float32)


def fractal_dem_torch(n_y: int, n_x: int, beta: float = 2.0, tilt: float = 0.01,
                      seed: int = 0, dx: float = 30.0, jitter: float = JITTER_M,
                      device: str = "cuda"):
    """Same recipe drawn with torch (complex64) on ``device`` for large grids."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    ky = torch.fft.fftfreq(n_y, device=device, dtype=torch.float32) * n_y
    kx = torch.fft.fftfreq(n_x, device=device, dtype=torch.float32) * n_x
    amp = torch.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    amp[0, 0] = 1.0
    amp.pow_(-beta / 2.0)
    amp[0, 0] = 0.0
    modes = torch.complex(torch.randn(n_y, n_x, generator=g, device=device),
                          torch.randn(n_y, n_x, generator=g, device=device))
    modes.mul_(amp)
    del amp
    z = torch.fft.ifft2(modes).real.contiguous()
    del modes
    lo, hi = z.min(), z.max()
    z.sub_(lo).mul_(Z_RANGE_M / float(hi - lo))
    if tilt:
        z.add_((tilt * dx) * (n_x - 1 - torch.arange(n_x, device=device,
                                                      dtype=torch.float32))[None, :])
    if jitter:
        z.add_(torch.rand(n_y, n_x, generator=g, device=device) * jitter)
    return z.to(torch.float32)


def rain_field(n_y: int, n_x: int, seed: int) -> np.ndarray:
    """Rain per cell, U[0, 1) float32, drawn from ``seed + 1``."""
    rng = np.random.default_rng(seed + 1)
    return rng.random((n_y, n_x), dtype=np.float32)


def rain_field_torch(n_y: int, n_x: int, seed: int, device: str = "cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed + 1)
    return torch.rand(n_y, n_x, generator=g, device=device, dtype=torch.float32)


def planar_dem(n_y: int, n_x: int, tilt: float = 0.01, dx: float = 30.0) -> np.ndarray:
    """Pure plane z = t * dx * (nx - 1 - x), float32 (no fractal, no jitter)."""
    z = tilt * dx * (n_x - 1 - np.arange(n_x, dtype=np.float64))
    return np.broadcast_to(z[None, :], (n_y, n_x)).astype(np.float32)


@dataclass
class TileSpec:
    n_y: int
    n_x: int
    beta: float
    seed: int


def batch_specs(count: int = 512, side_min: int = 64, side_max: int = 2048,
                beta_lo: float = 1.8, beta_hi: float = 2.4, seed: int = 0):
    """Tile sides log-uniform in [side_min, side_max], beta uniform, one seed
    per tile (``seed * 100003 + i``)."""
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(math.log(side_min), math.log(side_max), size=count))
    sides = np.clip(np.rint(sides).astype(np.int64), side_min, side_max)
    betas = rng.uniform(beta_lo, beta_hi, size=count)
    return [TileSpec(int(s), int(s), float(b), int(seed * 100003 + i))
            for i, (s, b) in enumerate(zip(sides, betas))]
