"""Independent solvers used to pin the oracle (test helpers; neither the oracle nor the CUDA path uses them).

* ``dst_poisson``: the discrete Poisson problem sum_{6 nb}(u_nb) - 6 u = h^2 4 pi G rho on the interior with
  Dirichlet data in the face ghosts, solved exactly by diagonalising the zero-Dirichlet 7-point operator with
  the type-I discrete sine transform (eigenvalues -4 sum_axes sin^2(p pi / (2 (n+1)))), scipy.fft.dstn.
* ``robin_poisson``: the same equation with the face ghosts eliminated through the static Robin relation
  r_g phi_g = r_i phi_i, assembled as a scipy.sparse matrix and solved with spsolve.
* ``green_sum``: the free-space solution of Poisson's equation (Sec. 1, Eq. Poissoneq.) for cell masses
  rho h^3, phi(x) = -G sum_j m_j / |x - x_j|, with the self term of a cell taken as -G rho h^2 C_cube,
  C_cube = integral over the unit cube of 1/|r| (computed here by Gauss-Legendre quadrature).
* ``analytic_sphere``: -2 pi G rho (R^2 - r^2/3) inside, -G M / r outside, M = 4 pi R^3 rho / 3.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sf
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def dst_poisson(h: float, G: float, rho: np.ndarray, ghosts: np.ndarray) -> np.ndarray:
    rhs = h * h * 4.0 * np.pi * G * np.array(rho, dtype=np.float64)
    P = ghosts
    rhs[:, :, 0] -= P[1:-1, 1:-1, 0]
    rhs[:, :, -1] -= P[1:-1, 1:-1, -1]
    rhs[:, 0, :] -= P[1:-1, 0, 1:-1]
    rhs[:, -1, :] -= P[1:-1, -1, 1:-1]
    rhs[0, :, :] -= P[0, 1:-1, 1:-1]
    rhs[-1, :, :] -= P[-1, 1:-1, 1:-1]
    nz, ny, nx = rho.shape
    lx = -4.0 * np.sin(np.arange(1, nx + 1) * np.pi / (2 * (nx + 1))) ** 2
    ly = -4.0 * np.sin(np.arange(1, ny + 1) * np.pi / (2 * (ny + 1))) ** 2
    lz = -4.0 * np.sin(np.arange(1, nz + 1) * np.pi / (2 * (nz + 1))) ** 2
    lam = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
    return sf.idstn(sf.dstn(rhs, type=1) / lam, type=1)


def robin_poisson(h: float, G: float, origin, rho: np.ndarray) -> np.ndarray:
    nz, ny, nx = rho.shape
    N = nx * ny * nz

    def idx(i, j, k):
        return (k * ny + j) * nx + i

    def centre(i, j, k):
        return np.array([origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h, origin[2] + (k + 0.5) * h])

    rows, cols, vals = [], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                q = idx(i, j, k)
                diag = -6.0
                for d, (di, dj, dk) in enumerate(((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))):
                    a, b, c = i + di, j + dj, k + dk
                    if 0 <= a < nx and 0 <= b < ny and 0 <= c < nz:
                        rows.append(q)
                        cols.append(idx(a, b, c))
                        vals.append(1.0)
                    else:  # ghost: phi_g = phi_i r_i / r_g
                        diag += np.linalg.norm(centre(i, j, k)) / np.linalg.norm(centre(a, b, c))
                rows.append(q)
                cols.append(q)
                vals.append(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    rhs = (h * h * 4.0 * np.pi * G * rho).reshape(-1)
    return spla.spsolve(A.tocsc(), rhs).reshape(nz, ny, nx)


def cube_inverse_distance_integral(order: int = 48) -> float:
    """C_cube = int_{[-1/2,1/2]^3} dV / |r|, by splitting into 24 congruent pyramids: one pyramid
    {0 <= y, z <= x <= 1/2} in coordinates x, y = x u, z = x v gives int_0^{1/2} x dx int_0^1 int_0^1 du dv /
    sqrt(1 + u^2 + v^2)."""
    t, w = np.polynomial.legendre.leggauss(order)
    u = 0.5 * (t + 1.0)
    wu = 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    inner = np.sum(wu[:, None] * wu[None, :] / np.sqrt(1.0 + U * U + V * V))
    return 24.0 * inner * 0.125  # int_0^{1/2} x dx = 1/8


def green_sum(points: np.ndarray, centres: np.ndarray, masses: np.ndarray, G: float, h: float,
              rho_self: np.ndarray | None = None) -> np.ndarray:
    """phi at points (P,3) from point masses at centres (M,3); where a point coincides with a centre the
    self term -G rho h^2 C_cube replaces the singular one (rho_self gives rho for each point)."""
    C = cube_inverse_distance_integral()
    out = np.zeros(len(points))
    for s in range(0, len(points), 256):
        p = points[s:s + 256]
        d = np.linalg.norm(p[:, None, :] - centres[None, :, :], axis=2)
        same = d < 1e-12 * h
        inv = np.where(same, 0.0, 1.0 / np.where(same, 1.0, d))
        out[s:s + 256] = -G * (inv @ masses)
        if rho_self is not None:
            out[s:s + 256] += np.where(same.any(axis=1), -G * rho_self[s:s + 256] * h * h * C, 0.0)
    return out


def analytic_sphere(X, Y, Z, R: float = 0.25, rho0: float = 1.0, G: float = 1.0):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    M = 4.0 * np.pi / 3.0 * R ** 3 * rho0
    return np.where(r < R, -2.0 * np.pi * G * rho0 * (R * R - r * r / 3.0), -G * M / np.maximum(r, 1e-300))
