"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and evaluates density fields; it holds none of the scheme's arithmetic (no
stencil, boundary condition, moment or norm), so both the CUDA path and the CPU oracle can take their inputs from
it.  The paper's own workloads (polytropes evolved by an MHD code, Sec. 2) are not reproducible here; these
analytic densities stand in for them with the shapes its tests have: a compact, centrally concentrated mass in
a box about twice its size, a perturbed 3D star, and two bodies moving through the grid.

Recipes (unit cube [-1/2, 1/2]^3, N cells per side, cell-centred):
  sphere       rho = 1 for r < 0.25, cell-averaged over 4^3 sub-cell centres.
  blobs        Gaussian blobs rho = A exp(-|x - c|^2 / (2 sigma^2)); sigma ~ U[0.02, 0.08], peak A ~ U[0.1, 2],
               centres uniform in the ball |c| < 0.3 (rejection from the cube), numpy PCG64 with the given seed.
  orbit        two blobs of sigma 0.05 and mass 1 each (peak 1/((2 pi)^{3/2} sigma^3)) at +-0.15 on a circle in
               the z = 0 plane, angle omega t with omega = 2 pi.
  noise        i.i.d. uniform values for stencil-parity inputs (the stencil is checked on arbitrary data).
"""
from __future__ import annotations

import numpy as np


def cell_centres_1d(n: int, lo: float = -0.5, h: float | None = None) -> np.ndarray:
    h = 1.0 / n if h is None else h
    return lo + (np.arange(n) + 0.5) * h


def sphere_density(nx: int, ny: int | None = None, nz: int | None = None, radius: float = 0.25,
                   rho0: float = 1.0, sub: int = 4, h: float | None = None, lo: float = -0.5) -> np.ndarray:
    """Uniform sphere at the origin, cell-averaged by sub^3 point sampling.  Shape (nz, ny, nx), float64."""
    ny = ny or nx
    nz = nz or nx
    h = 1.0 / nx if h is None else h
    offs = ((np.arange(sub) + 0.5) / sub - 0.5) * h
    xs = cell_centres_1d(nx, lo, h)
    ys = cell_centres_1d(ny, lo, h)
    zs = cell_centres_1d(nz, lo, h)
    frac = np.zeros((nz, ny, nx))
    r2max = radius * radius
    for oz in offs:
        z2 = (zs + oz) ** 2
        for oy in offs:
            y2 = (ys + oy) ** 2
            for ox in offs:
                x2 = (xs + ox) ** 2
                frac += (z2[:, None, None] + y2[None, :, None] + x2[None, None, :]) < r2max
    return rho0 * frac / sub ** 3


def draw_blobs(count: int, seed: int, sigma=(0.02, 0.08), amp=(0.1, 2.0), ball: float = 0.3) -> np.ndarray:
    """(count, 5) array of (cx, cy, cz, sigma, peak) drawn with numpy's PCG64 from the seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 5))
    for b in range(count):
        while True:
            c = rng.uniform(-ball, ball, size=3)
            if c @ c < ball * ball:
                break
        out[b, :3] = c
        out[b, 3] = rng.uniform(*sigma)
        out[b, 4] = rng.uniform(*amp)
    return out


def blob_density(nx: int, blobs: np.ndarray, ny: int | None = None, nz: int | None = None,
                 h: float | None = None, lo: float = -0.5) -> np.ndarray:
    """Sum of Gaussian blobs (rows of (cx, cy, cz, sigma, peak)) at cell centres.  Shape (nz, ny, nx)."""
    ny = ny or nx
    nz = nz or nx
    h = 1.0 / nx if h is None else h
    xs = cell_centres_1d(nx, lo, h)
    ys = cell_centres_1d(ny, lo, h)
    zs = cell_centres_1d(nz, lo, h)
    rho = np.zeros((nz, ny, nx))
    for cxb, cyb, czb, s, a in blobs:
        ex = np.exp(-((xs - cxb) ** 2) / (2 * s * s))
        ey = np.exp(-((ys - cyb) ** 2) / (2 * s * s))
        ez = np.exp(-((zs - czb) ** 2) / (2 * s * s))
        rho += a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return rho


def orbit_blobs(t: float, radius: float = 0.15, sigma: float = 0.05, mass: float = 1.0,
                omega: float = 2.0 * np.pi) -> np.ndarray:
    """Two equal blobs on a circular orbit in the z = 0 plane at time t, as rows of (cx, cy, cz, sigma, peak)."""
    peak = mass / ((2.0 * np.pi) ** 1.5 * sigma ** 3)
    ang = omega * t
    c, s = np.cos(ang), np.sin(ang)
    return np.array([[radius * c, radius * s, 0.0, sigma, peak],
                     [-radius * c, -radius * s, 0.0, sigma, peak]])


def noise(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform field (float64) from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def probes(count: int, seed: int, ball: float = 0.4) -> np.ndarray:
    """(count, 3) points uniform in the ball |x| < ball (rejection from the cube)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((count, 3))
    for p in range(count):
        while True:
            c = rng.uniform(-ball, ball, size=3)
            if c @ c < ball * ball:
                break
        out[p] = c
    return out


def batch_sides(count: int, seed: int, choices=(64, 96, 128, 160, 192)) -> np.ndarray:
    """Side lengths of the independent grids of the batching workload, uniform over the choices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(np.asarray(choices), size=count)


def batch_blob_counts(count: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return rng.integers(1, 7, size=count)


def blob_density_torch(nx: int, blobs: np.ndarray, device, dtype, ny: int | None = None, nz: int | None = None,
                       h: float | None = None, lo: float = -0.5):
    """The same field as blob_density, evaluated with torch on a device (for large benchmark inputs)."""
    import torch

    ny = ny or nx
    nz = nz or nx
    h = 1.0 / nx if h is None else h
    f64 = torch.float64
    xs = lo + (torch.arange(nx, device=device, dtype=f64) + 0.5) * h
    ys = lo + (torch.arange(ny, device=device, dtype=f64) + 0.5) * h
    zs = lo + (torch.arange(nz, device=device, dtype=f64) + 0.5) * h
    rho = torch.zeros((nz, ny, nx), device=device, dtype=dtype)
    for cxb, cyb, czb, s, a in blobs:
        ex = torch.exp(-((xs - cxb) ** 2) / (2 * s * s))
        ey = torch.exp(-((ys - cyb) ** 2) / (2 * s * s))
        ez = torch.exp(-((zs - czb) ** 2) / (2 * s * s))
        rho += (a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).to(dtype)
    return rho
