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
  polytrope    the 3D star of the paper's virial test (Sec. 2): a Lane-Emden polytrope of index n (default 3)
               with mass M and radius R at the origin, point-sampled at cell centres, v = 0, P = K rho^(1+1/n),
               plus a dilute isothermal atmosphere in hydrostatic equilibrium with the star's potential (density
               atm * rho_c at the surface, sound speed squared atm_kt * G M / R), optional i.i.d. relative density
               perturbations inside the star, and the star's exact potential for seeding phi.
  hydro states primitive fields (rho, vx, vy, vz, P): shock tubes along an axis and i.i.d. bounded noise.
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


def lane_emden(n: float, dxi: float = 1e-3):
    """Lane-Emden function of index n: (1/xi^2) d/dxi (xi^2 dtheta/dxi) = -theta^n, theta(0) = 1, theta'(0) = 0.

    Classical RK4 in (theta, theta') with step dxi from the series start theta = 1 - xi^2/6 + n xi^4/120 at
    xi = dxi, up to the first zero xi_1 (refined by Newton steps on the last RK4 step), or to xi = 20 when there is
    none (n >= 5).  Returns (xi, theta, dtheta, xi1, omega) with omega = -xi1^2 theta'(xi1) (nan without a zero).
    """
    def rhs(x, t, dt):
        return dt, -(max(t, 0.0) ** n) - 2.0 * dt / x

    x = dxi
    t = 1.0 - x * x / 6.0 + n * x ** 4 / 120.0
    d = -x / 3.0 + n * x ** 3 / 30.0
    xs, ts, ds = [0.0, x], [1.0, t], [0.0, d]

    def rk4(x, t, d, hh):
        k1 = rhs(x, t, d)
        k2 = rhs(x + hh / 2, t + hh / 2 * k1[0], d + hh / 2 * k1[1])
        k3 = rhs(x + hh / 2, t + hh / 2 * k2[0], d + hh / 2 * k2[1])
        k4 = rhs(x + hh, t + hh * k3[0], d + hh * k3[1])
        return (t + hh / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
                d + hh / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))

    while x < 20.0:
        tn, dn = rk4(x, t, d, dxi)
        if tn <= 0.0:
            hh = -t / d
            for _ in range(4):  # Newton on theta(x + hh) = 0 along the RK4 step
                tz, dz = rk4(x, t, d, hh)
                hh -= tz / dz
            tz, dz = rk4(x, t, d, hh)
            xs.append(x + hh)
            ts.append(0.0)
            ds.append(dz)
            xi1 = x + hh
            return np.array(xs), np.array(ts), np.array(ds), xi1, -xi1 * xi1 * dz
        x, t, d = x + dxi, tn, dn
        xs.append(x)
        ts.append(t)
        ds.append(d)
    return np.array(xs), np.array(ts), np.array(ds), float("nan"), float("nan")


def _hermite(xs, ts, ds, x):
    """Cubic Hermite interpolation of theta from the RK4 table (values and derivatives) at points x <= xs[-1]."""
    x = np.asarray(x, dtype=np.float64)
    k = np.clip(np.searchsorted(xs, x, side="right") - 1, 0, len(xs) - 2)
    x0, x1 = xs[k], xs[k + 1]
    w = x1 - x0
    s = (x - x0) / w
    h00 = (1 + 2 * s) * (1 - s) ** 2
    h10 = s * (1 - s) ** 2
    h01 = s * s * (3 - 2 * s)
    h11 = s * s * (s - 1)
    return h00 * ts[k] + h10 * w * ds[k] + h01 * ts[k + 1] + h11 * w * ds[k + 1]


def polytrope(nx: int, n_index: float = 3.0, mass: float = 1.0, radius: float = 1.0 / 3.0, G: float = 1.0,
              atm: float = 1e-6, atm_kt: float = 0.5, pert: float = 0.0, seed: int = 0, ny: int | None = None,
              nz: int | None = None, h: float | None = None, lo: float = -0.5):
    """Polytropic star at the origin: returns (rho, P, phi, info), each field (nz, ny, nx) float64.

    Star: rho_c theta^n(r / alpha) with alpha = R / xi_1 and rho_c = M / (4 pi alpha^3 omega); P = K rho^(1+1/n)
    with K = 4 pi G alpha^2 rho_c^(1-1/n) / (n+1); exact potential -G M / R - (n+1) K rho_c^(1/n) theta inside,
    -G M / r outside.
    Atmosphere (a "dilute atmosphere" of negligible mass, Sec. 2): an isothermal component with P_a = k_T rho_a,
    k_T = atm_kt G M / R, in hydrostatic equilibrium with that potential everywhere, rho_a = atm rho_c
    exp(-(phi - phi(R)) / k_T), added to the star's density and pressure (both components balance gravity on their
    own, so the sum does too, and the atmosphere does not fall onto the star).  atm = 0: no atmosphere.
    pert > 0 multiplies rho inside the star by 1 + pert u, u ~ U[-1, 1] from PCG64(seed) (P is left unchanged).
    phi is the star's potential; the atmosphere's own gravity (its mass is ~6e-4 M for the defaults) is left out.
    """
    ny = ny or nx
    nz = nz or nx
    h = 1.0 / nx if h is None else h
    xs_, ts_, ds_, xi1, omega = lane_emden(n_index)
    alpha = radius / xi1
    rho_c = mass / (4.0 * np.pi * alpha ** 3 * omega)
    K = 4.0 * np.pi * G * alpha ** 2 * rho_c ** (1.0 - 1.0 / n_index) / (n_index + 1.0)
    x = cell_centres_1d(nx, lo, h)
    y = cell_centres_1d(ny, lo, h)
    z = cell_centres_1d(nz, lo, h)
    r = np.sqrt(z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2)
    inside = r < radius
    theta = np.zeros_like(r)
    theta[inside] = np.maximum(_hermite(xs_, ts_, ds_, r[inside] / alpha), 0.0)
    rho = rho_c * theta ** n_index
    if pert > 0.0:
        u = noise(r.shape, seed, -1.0, 1.0)
        rho = np.where(inside, rho * (1.0 + pert * u), rho)
    P = K * (rho_c * theta ** n_index) ** (1.0 + 1.0 / n_index)
    phi = np.where(inside, -G * mass / radius - (n_index + 1.0) * K * rho_c ** (1.0 / n_index) * theta,
                   -G * mass / np.maximum(r, 1e-300))
    kt = atm_kt * G * mass / radius
    rho_a = atm * rho_c * np.exp(-(phi + G * mass / radius) / kt) if atm > 0.0 else np.zeros_like(r)
    rho = rho + rho_a
    P = P + kt * rho_a
    rho_min = float(rho_a.min()) if atm > 0.0 else 0.0
    info = dict(rho_c=rho_c, K=K, alpha=alpha, xi1=xi1, omega=omega, kt=kt, rho_atm=rho_min, p_atm=kt * rho_min,
                atm_mass=float(rho_a.sum()) * h ** 3)
    return rho, P, phi, info


def shock_tube(shape, axis: int, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), frac: float = 0.5):
    """Primitive fields (5, nz, ny, nx) of a Riemann problem along axis (0 = x, 1 = y, 2 = z): (rho, u_n, P) on
    the cells below frac of the axis length, the right triple above, transverse velocities zero."""
    nz, ny, nx = shape
    n = (nx, ny, nz)[axis]
    side = (np.arange(n) + 0.5) < frac * n
    W = np.zeros((5,) + tuple(shape))
    for q, (a, b) in ((0, (left[0], right[0])), (1 + axis, (left[1], right[1])), (4, (left[2], right[2]))):
        line = np.where(side, a, b)
        W[q] = line.reshape([(n if ax == axis else 1) for ax in (2, 1, 0)])
    return W


def hydro_noise(shape, seed: int, drho=0.5, dv=0.3, dp=0.5):
    """Primitive fields (5, nz, ny, nx): rho = 1 + drho u, v_i = dv u, P = 1 + dp u with independent i.i.d.
    u ~ U[-1, 1] (PCG64 from seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-1.0, 1.0, size=(5,) + tuple(shape))
    return np.stack([1.0 + drho * u[0], dv * u[1], dv * u[2], dv * u[3], 1.0 + dp * u[4]])
