"""Seeded synthetic inputs for the thin-disk force solve.

This module holds input recipes only (densities, random weights, sample points); none of
the force method's arithmetic lives here.  It is the one module that both the oracle-side
tests and the GPU-side bench/tests import, so that both sides see identical inputs.

Recipes (cell centres x_i = lo + (i + 1/2) dx on [lo, hi]^2, axis 0 is x):
  * generalized Maclaurin disk D_n: sigma_0 (1 - R^2/a^2)^(n - 1/2) for R < a (Sec. 3);
  * perturbed disk: D_n x (1 + 0.1 g), g a Gaussian random field of correlation length
    0.02 (white N(0,1) filtered by a Gaussian of std 0.02/sqrt(2), renormalised to unit
    sample std), clipped at 0 and zeroed for R >= a;
  * clumps: 64 Gaussians, centres uniform in radius (< 0.4) and angle, widths
    U(0.005, 0.05), amplitudes LogNormal(0, 1), in physical coordinates on [-0.5, 0.5]^2;
  * batched uneven set: 256 grids with Nx, Ny drawn from {128, ..., 1024}, order from
    {1, 2, 3}, each with its own clump field (seed 4000 + d);
  * adjoint weights g_x, g_y ~ N(0, 1) and finite-difference probe points.
"""
from __future__ import annotations

import numpy as np

BATCH_SIZES = (128, 192, 256, 384, 512, 768, 1024)


def cell_centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def grid(nx: int, ny: int, lo: float = -0.5, hi: float = 0.5):
    x = cell_centres(nx, lo, hi)
    y = cell_centres(ny, lo, hi)
    return x, y, (hi - lo) / nx, (hi - lo) / ny


def maclaurin_density(n: int, x: np.ndarray, y: np.ndarray, a: float, sigma0: float = 1.0):
    X, Y = np.meshgrid(x, y, indexing="ij")
    s = 1.0 - (X * X + Y * Y) / (a * a)
    out = np.zeros_like(s)
    inside = s > 0.0
    out[inside] = sigma0 * s[inside] ** (n - 0.5)
    return out


def gaussian_random_field(nx: int, ny: int, dx: float, dy: float, ell: float, seed: int):
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((nx, ny))
    std = ell / np.sqrt(2.0)
    kx = np.fft.fftfreq(nx, d=dx)
    ky = np.fft.rfftfreq(ny, d=dy)
    filt = np.exp(-2.0 * np.pi ** 2 * std ** 2 * (kx[:, None] ** 2 + ky[None, :] ** 2))
    g = np.fft.irfft2(np.fft.rfft2(white) * filt, s=(nx, ny))
    g -= g.mean()
    return g / g.std()


def perturbed_disk(n: int, N: int, seed: int = 2, a: float = 0.4, amp: float = 0.1,
                   ell: float = 0.02):
    x, y, dx, dy = grid(N, N)
    base = maclaurin_density(n, x, y, a)
    g = gaussian_random_field(N, N, dx, dy, ell, seed)
    out = np.clip(base * (1.0 + amp * g), 0.0, None)
    X, Y = np.meshgrid(x, y, indexing="ij")
    out[X * X + Y * Y >= a * a] = 0.0
    return out


def clumps(nx: int, ny: int, seed: int, count: int = 64, rmax: float = 0.4):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, rmax, count)
    th = rng.uniform(0.0, 2.0 * np.pi, count)
    w = rng.uniform(0.005, 0.05, count)
    amp = rng.lognormal(0.0, 1.0, count)
    x, y, _, _ = grid(nx, ny)
    out = np.zeros((nx, ny))
    for c in range(count):
        xc, yc = r[c] * np.cos(th[c]), r[c] * np.sin(th[c])
        gx = np.exp(-((x - xc) ** 2) / (2.0 * w[c] ** 2))
        gy = np.exp(-((y - yc) ** 2) / (2.0 * w[c] ** 2))
        out += amp[c] * np.outer(gx, gy)
    return out


def batched_specs(count: int = 256, seed: int = 4):
    """(nx, ny, order, field seed) for each grid of the uneven batch."""
    rng = np.random.default_rng(seed)
    nx = rng.choice(BATCH_SIZES, count)
    ny = rng.choice(BATCH_SIZES, count)
    order = rng.integers(1, 4, count)
    return [(int(nx[d]), int(ny[d]), int(order[d]), seed * 1000 + d) for d in range(count)]


def adjoint_weights(nx: int, ny: int, seed: int = 6):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))


def fd_points(nx: int, ny: int, seed: int = 7, rdisk: float = 0.4):
    """32 probe cells: 16 uniform, 8 inside R < rdisk, 8 on the edge rows/columns."""
    rng = np.random.default_rng(seed)
    pts = [(int(rng.integers(nx)), int(rng.integers(ny))) for _ in range(16)]
    x, y, _, _ = grid(nx, ny)
    while len(pts) < 24:
        i, j = int(rng.integers(nx)), int(rng.integers(ny))
        if x[i] ** 2 + y[j] ** 2 < rdisk ** 2:
            pts.append((i, j))
    for e in range(8):
        side = e % 4
        t = int(rng.integers(min(nx, ny)))
        pts.append([(0, t), (nx - 1, t), (t, 0), (t, ny - 1)][side])
    return pts


def sample_points(nx: int, ny: int, count: int, seed: int):
    """Output cells for sampled parity at full size: corners, edges and random cells."""
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, ny // 2)]
    while len(pts) < count:
        pts.append((int(rng.integers(nx)), int(rng.integers(ny))))
    return pts
