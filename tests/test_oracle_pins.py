"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself, chosen so that a dropped term, a wrong sign,
a wrong coefficient or a transposed index in the oracle fails at least one of them:

* fixed point = discrete Poisson solution (DST-I solve)          -> stencil, source sign and 4 pi G, Dirichlet
* exact discrete plane wave of the leapfrog scheme (periodic)    -> time integrator, nu^2, wrap, mean removal
* analytic uniform sphere, convergence with h                    -> the whole steady state vs Eq. Poissoneq.
* brute-force Green's-function sum on 16^3                       -> multipole ghosts and the Robin steady state
* sparse direct solve with the static Robin relation             -> Robin ghost update's fixed point
* spherical-harmonic addition theorem and textbook Y_00, Y_10    -> the harmonic basis of the moments
* point-mass multipole truncation bound                          -> moments + expansion
* quadratic potential                                            -> central-difference gradient, residual
* linearity in rho                                               -> every boundary mode
* central finite differences (exact for a quadratic loss) and the dot-product test -> discrete adjoint
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle as O
from paper_1602_05700_gb300 import inputs as I
from tests import poisson_ref as R


def _grid(nx, ny, nz, h, bc, c=1.0, G=1.0, cfl=0.5):
    origin = (-0.5 * nx * h, -0.5 * ny * h, -0.5 * nz * h)
    return O.Grid(nx, ny, nz, h, origin, c, G, cfl * h / (c * np.sqrt(3.0)), bc)


# ---- fixed point --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(12, 10, 14), (7, 9, 5)])
def test_fixed_point_is_discrete_poisson_solution(shape):
    nx, ny, nz = shape
    g = _grid(nx, ny, nz, 0.07, O.BC_DIRICHLET, c=1.3, G=0.7)
    rho = I.noise(g.shape, 11, 0.0, 2.0)
    ghosts = O.ghosted(g)
    data = I.noise(g.ghosted_shape, 12, -3.0, -1.0)
    for sl in ((slice(1, -1), slice(1, -1), 0), (slice(1, -1), slice(1, -1), -1), (slice(1, -1), 0, slice(1, -1)),
               (slice(1, -1), -1, slice(1, -1)), (0, slice(1, -1), slice(1, -1)), (-1, slice(1, -1), slice(1, -1))):
        ghosts[sl] = data[sl]
    u = R.dst_poisson(g.h, g.G, rho, ghosts)
    # the DST solution satisfies the discrete equation (checked here without the oracle)
    full = ghosts.copy()
    full[1:-1, 1:-1, 1:-1] = u
    lap = (full[1:-1, 1:-1, :-2] + full[1:-1, 1:-1, 2:] + full[1:-1, :-2, 1:-1] + full[1:-1, 2:, 1:-1]
           + full[:-2, 1:-1, 1:-1] + full[2:, 1:-1, 1:-1] - 6 * u) / g.h ** 2
    assert np.abs(lap - 4 * np.pi * g.G * rho).max() < 1e-9 * np.abs(4 * np.pi * g.G * rho).max()
    phi = full.copy()
    prev = full.copy()
    O.run(g, phi, prev, rho, 200)
    assert np.abs(phi[1:-1, 1:-1, 1:-1] - u).max() < 1e-12 * np.abs(u).max()
    # and the boundary data is untouched
    assert np.array_equal(phi[0, 1:-1, 1:-1], ghosts[0, 1:-1, 1:-1])
    # a state off the fixed point does move (the check above is not vacuous)
    phi2 = full.copy()
    phi2[1:-1, 1:-1, 1:-1] *= 1.01
    prev2 = phi2.copy()
    O.run(g, phi2, prev2, rho, 5)
    assert np.abs(phi2[1:-1, 1:-1, 1:-1] - 1.01 * u).max() > 1e-6 * np.abs(u).max()


# ---- exact discrete plane wave -----------------------------------------------------------------------------

@pytest.mark.parametrize("modes", [(1, 0, 0), (2, 1, 3), (0, 5, 2)])
def test_plane_wave_dispersion_periodic(modes):
    nx, ny, nz = 16, 12, 20
    g = _grid(nx, ny, nz, 0.05, O.BC_PERIODIC, c=2.0, cfl=0.9)
    X, Y, Z = g.centres()
    L = np.array([nx, ny, nz]) * g.h
    k = 2 * np.pi * np.array(modes) / L
    nu = g.c * g.dt / g.h
    cos_w = 1 - 2 * nu ** 2 * np.sum(np.sin(k * g.h / 2) ** 2)
    w = np.arccos(cos_w)  # omega * dt
    kx = k[0] * X + k[1] * Y + k[2] * Z
    rho = np.zeros(g.shape)
    phi, prev = O.initial_state(g, rho, phi0=np.cos(kx), phi_prev0=np.cos(kx + w))
    n = 300
    O.run(g, phi, prev, rho, n)
    exact = np.cos(kx - n * w)
    assert np.abs(phi[1:-1, 1:-1, 1:-1] - exact).max() < 2e-11
    # group/phase speed tends to c for long waves: omega/|k| -> c
    if modes == (1, 0, 0):
        assert abs(w / g.dt / np.linalg.norm(k) - g.c) < 0.01 * g.c


def test_periodic_source_uses_mean_subtracted_density():
    g = _grid(8, 8, 8, 0.1, O.BC_PERIODIC)
    rho = np.full(g.shape, 5.0)
    phi, prev = O.initial_state(g, rho)
    O.run(g, phi, prev, rho, 50)
    assert np.abs(phi).max() < 1e-12


# ---- the uniform sphere (steady state vs Eq. Poissoneq.) ---------------------------------------------------

def test_sphere_dirichlet_monopole_converges_to_analytic():
    errs = []
    for n in (16, 32, 48):
        g = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
        rho = I.sphere_density(n)
        phi, prev = O.initial_state(g, rho, lmax=0)
        # the monopole ghosts are -G M / r with the discrete mass
        M = O.mass(g, rho)
        Xg, Yg, Zg = g.centres(ghosts=True)
        rg = np.sqrt(Xg[0, 1:-1, 1:-1] ** 2 + Yg[0, 1:-1, 1:-1] ** 2 + Zg[0, 1:-1, 1:-1] ** 2)
        assert np.allclose(phi[0, 1:-1, 1:-1], -g.G * M / rg, rtol=1e-12, atol=0)
        u = R.dst_poisson(g.h, g.G, rho, phi)
        phi[1:-1, 1:-1, 1:-1] = u
        prev[:] = phi
        O.run(g, phi, prev, rho, 40)
        assert np.abs(phi[1:-1, 1:-1, 1:-1] - u).max() < 1e-12 * np.abs(u).max()
        X, Y, Z = g.centres()
        an = R.analytic_sphere(X, Y, Z)
        errs.append(np.sqrt(np.mean((u - an) ** 2) / np.mean(an ** 2)))
    assert errs[0] < 1e-2 and errs[1] < 2e-3 and errs[2] < 6e-4
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 3.0  # close to second order


def test_sphere_robin_relaxes_to_analytic():
    n = 16
    g = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN)
    rho = I.sphere_density(n)
    phi, prev = O.initial_state(g, rho)
    steps = 0
    change = 1.0
    while change > 1e-10 and steps < 20000:
        O.run(g, phi, prev, rho, 250)
        steps += 250
        change = np.abs(phi - prev).max() / np.abs(phi).max()
    assert change <= 1e-10
    X, Y, Z = g.centres()
    an = R.analytic_sphere(X, Y, Z)
    u = phi[1:-1, 1:-1, 1:-1]
    assert np.sqrt(np.mean((u - an) ** 2) / np.mean(an ** 2)) < 1e-2
    # the mass of the 4^3-subsampled sphere is the analytic one to the sampling error
    assert abs(O.mass(g, rho) - np.pi / 48) < 0.01 * np.pi / 48


def test_robin_steady_state_matches_sparse_solve():
    g = _grid(10, 12, 11, 0.1, O.BC_ROBIN)
    blobs = np.array([[0.05, -0.03, 0.02, 0.12, 1.5], [-0.1, 0.08, -0.05, 0.1, 0.8]])
    X, Y, Z = g.centres()
    rho = np.zeros(g.shape)
    for cxb, cyb, czb, s, a in blobs:
        rho += a * np.exp(-((X - cxb) ** 2 + (Y - cyb) ** 2 + (Z - czb) ** 2) / (2 * s * s))
    ref = R.robin_poisson(g.h, g.G, g.origin, rho)
    phi, prev = O.initial_state(g, rho)
    for _ in range(200):
        O.run(g, phi, prev, rho, 500)
        if np.abs(phi - prev).max() < 1e-13 * np.abs(phi).max():
            break
    u = phi[1:-1, 1:-1, 1:-1]
    assert np.abs(u - ref).max() < 1e-9 * np.abs(ref).max()
    # the ghosts sit at the static Robin relation r_g phi_g = r_i phi_i
    Xg, Yg, Zg = g.centres(ghosts=True)
    rg = np.sqrt(Xg ** 2 + Yg ** 2 + Zg ** 2)
    assert np.allclose(rg[1:-1, 1:-1, 0] * phi[1:-1, 1:-1, 0], rg[1:-1, 1:-1, 1] * phi[1:-1, 1:-1, 1], rtol=1e-9)


def test_robin_ghost_update_consistent_with_radiation_condition():
    """Manufactured outgoing monopole wave phi = f(r - c t) / r satisfies d_t(r phi) + c d_r(r phi) = 0 exactly.
    One sub-step of the ghost update, started from the exact wave, must reproduce the exact increment of r phi
    at the ghosts to first order in h (upwind), on every face and at oblique incidence."""
    errs = []
    for n in (16, 32, 64):
        g = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN)
        Xg, Yg, Zg = g.centres(ghosts=True)
        r = np.sqrt(Xg ** 2 + Yg ** 2 + Zg ** 2)

        def f(s):
            return np.exp(-(s - 0.55) ** 2 / (2 * 0.1 ** 2))

        phi = f(r) / r
        prev = f(r + g.c * g.dt) / r
        out = O.step(g, phi, prev, np.zeros(g.shape))
        exact = f(r - g.c * g.dt) / r
        worst = 0.0
        for sl in ((slice(1, -1), slice(1, -1), 0), (slice(1, -1), slice(1, -1), -1), (slice(1, -1), 0, slice(1, -1)),
                   (slice(1, -1), -1, slice(1, -1)), (0, slice(1, -1), slice(1, -1)), (-1, slice(1, -1), slice(1, -1))):
            d_num = out[sl] - phi[sl]
            d_ex = exact[sl] - phi[sl]
            worst = max(worst, np.abs(d_num - d_ex).max() / np.abs(d_ex).max())
        errs.append(worst)
    assert errs[2] < 0.12
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_robin_absorbs_outgoing_pulse():
    """An outgoing pulse leaves a Robin box (Sec. 4: errors propagate out of the boundary) but stays in a
    Dirichlet box (the leapfrog scheme is lossless)."""
    energies = {}
    for bc in (O.BC_ROBIN, O.BC_DIRICHLET):
        g = _grid(24, 24, 24, 1.0 / 24, bc)
        X, Y, Z = g.centres()
        pulse = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 0.05 ** 2))
        rho = np.zeros(g.shape)
        phi, prev = O.ghosted(g, pulse), O.ghosted(g, pulse)
        O.run(g, phi, prev, rho, 400)
        energies[bc] = np.sum(phi[1:-1, 1:-1, 1:-1] ** 2)
    assert energies[O.BC_ROBIN] < 0.05 * energies[O.BC_DIRICHLET]


# ---- Green's-function sum ------------------------------------------------------------------------------------

def test_green_sum_16cubed():
    n = 16
    g = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    blobs = np.array([[0.04, -0.02, 0.03, 0.09, 1.0], [-0.05, 0.03, -0.02, 0.08, 0.7]])
    rho = I.blob_density(n, blobs)
    X, Y, Z = g.centres()
    centres = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    masses = rho.ravel() * g.h ** 3
    # (a) multipole ghosts (l <= 4) against the brute-force sum at the ghost centres
    phi, _ = O.initial_state(g, rho, lmax=4)
    Xg, Yg, Zg = g.centres(ghosts=True)
    face = (slice(None), slice(1, -1), 0)
    pts = np.stack([Xg[1:-1, 1:-1, 0].ravel(), Yg[1:-1, 1:-1, 0].ravel(), Zg[1:-1, 1:-1, 0].ravel()], axis=1)
    gs = R.green_sum(pts, centres, masses, g.G, g.h)
    assert np.abs(phi[1:-1, 1:-1, 0].ravel() - gs).max() < 2e-4 * np.abs(gs).max()
    # monopole-only ghosts are visibly worse than l <= 4 (the moments carry the shape)
    phi0, _ = O.initial_state(g, rho, lmax=0)
    assert np.abs(phi0[1:-1, 1:-1, 0].ravel() - gs).max() > 3 * np.abs(phi[1:-1, 1:-1, 0].ravel() - gs).max()
    # (b) interior: the Robin steady state of the scheme approaches the free-space solution
    gr = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN)
    p, q = O.initial_state(gr, rho)
    for _ in range(80):
        O.run(gr, p, q, rho, 250)
        if np.abs(p - q).max() < 1e-11 * np.abs(p).max():
            break
    gi = R.green_sum(centres, centres, masses, g.G, g.h, rho_self=rho.ravel()).reshape(g.shape)
    u = p[1:-1, 1:-1, 1:-1]
    assert np.sqrt(np.mean((u - gi) ** 2) / np.mean(gi ** 2)) < 2e-2


# ---- harmonics and moments ------------------------------------------------------------------------------------

def test_real_harmonics_addition_theorem():
    rng = np.random.default_rng(5)
    lmax = 6
    for _ in range(10):
        a = rng.normal(size=3)
        b = rng.normal(size=3)
        Ya = O.real_ylm(lmax, *a)
        Yb = O.real_ylm(lmax, *b)
        cg = a @ b / np.linalg.norm(a) / np.linalg.norm(b)
        for l in range(lmax + 1):
            s = np.sum(Ya[l * l:(l + 1) ** 2] * Yb[l * l:(l + 1) ** 2])
            assert abs(s - (2 * l + 1) / (4 * np.pi) * eval_legendre(l, cg)) < 1e-12
    x, y, z = 0.3, -0.4, 0.5
    Y = O.real_ylm(1, x, y, z)
    r = np.sqrt(x * x + y * y + z * z)
    assert abs(Y[0] - 1 / np.sqrt(4 * np.pi)) < 1e-15
    assert abs(Y[2] - np.sqrt(3 / (4 * np.pi)) * z / r) < 1e-15
    assert abs(abs(Y[3]) - np.sqrt(3 / (4 * np.pi)) * abs(x) / r) < 1e-15
    assert abs(abs(Y[1]) - np.sqrt(3 / (4 * np.pi)) * abs(y) / r) < 1e-15


@pytest.mark.parametrize("lmax", [0, 2, 4, 6])
def test_multipole_point_mass_truncation(lmax):
    g = _grid(8, 8, 8, 0.125, O.BC_DIRICHLET, G=2.0)
    rho = np.zeros(g.shape)
    rho[5, 2, 6] = 3.0
    X, Y, Z = g.centres()
    x0 = np.array([X[5, 2, 6], Y[5, 2, 6], Z[5, 2, 6]])
    m = 3.0 * g.h ** 3
    Q = O.moments(g, rho, lmax)
    rng = np.random.default_rng(1)
    d0 = np.linalg.norm(x0)
    for _ in range(20):
        p = rng.normal(size=3)
        p *= rng.uniform(1.5, 4.0) / np.linalg.norm(p)
        r = np.linalg.norm(p)
        exact = -g.G * m / np.linalg.norm(p - x0)
        bound = g.G * m / (r - d0) * (d0 / r) ** (lmax + 1)
        assert abs(O.multipole_phi(g, lmax, Q, *p) - exact) <= bound * (1 + 1e-9) + 1e-15
    assert abs(Q[0] * np.sqrt(4 * np.pi) - m) < 1e-15


# ---- gradient and residual ------------------------------------------------------------------------------------

def test_accel_and_residual_exact_on_quadratic():
    g = _grid(9, 7, 8, 0.11, O.BC_DIRICHLET, G=0.5)
    Xg, Yg, Zg = g.centres(ghosts=True)
    a, b, c, d, e = 0.7, -1.3, 0.4, 2.1, -0.6
    phi = a * Xg ** 2 + b * Yg * Zg + c * Zg ** 2 + d * Xg + e * Yg
    ax, ay, az = O.accel(g, phi)
    X, Y, Z = g.centres()
    assert np.abs(ax + (2 * a * X + d)).max() < 1e-12
    assert np.abs(ay + (b * Z + e)).max() < 1e-12
    assert np.abs(az + (b * Y + 2 * c * Z)).max() < 1e-12
    lap = 2 * a + 2 * c
    rho = np.full(g.shape, lap / (4 * np.pi * g.G))
    rms, mx = O.residual(g, phi, rho)
    assert mx < 1e-10
    rho2 = np.zeros(g.shape)
    rms2, mx2 = O.residual(g, phi, rho2)
    assert abs(mx2 - abs(lap)) < 1e-10 and abs(rms2 - abs(lap)) < 1e-10


def test_compare_metrics():
    g = _grid(5, 4, 3, 0.2, O.BC_DIRICHLET)
    b = O.ghosted(g, -1.0 - I.noise(g.shape, 3, 0.0, 1.0))
    a = b * (1 + 1e-3)
    l2, linf, avg = O.compare(g, a, b)
    assert abs(l2 - 1e-3) < 1e-15 and abs(linf - 1e-3) < 1e-15 and abs(avg - 1e-3) < 1e-15


# ---- linearity ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bc,lmax", [(O.BC_ROBIN, 0), (O.BC_PERIODIC, 0), (O.BC_DIRICHLET, 4)])
def test_linearity_in_rho(bc, lmax):
    g = _grid(10, 9, 11, 0.1, bc)
    r1 = I.noise(g.shape, 21, 0.0, 1.0)
    r2 = I.noise(g.shape, 22, 0.0, 1.0)
    out = []
    for rho in (r1, r2, 2.5 * r1 - 1.5 * r2):
        phi, prev = O.initial_state(g, rho, lmax=lmax)
        O.run(g, phi, prev, rho, 40)
        out.append(phi[1:-1, 1:-1, 1:-1])
    comb = 2.5 * out[0] - 1.5 * out[1]
    assert np.abs(out[2] - comb).max() < 1e-12 * np.abs(comb).max()


# ---- discrete adjoint ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [O.BC_DIRICHLET, O.BC_ROBIN, O.BC_PERIODIC])
def test_adjoint_against_finite_differences(bc):
    g = _grid(8, 9, 10, 0.1, bc, cfl=0.8)
    T = 25
    rho = I.noise(g.shape, 31, 0.0, 1.0)
    w = I.noise(g.shape, 32, 0.0, 1.0)
    target = I.noise(g.shape, 33, -0.1, 0.1)

    def forward(r):
        phi, prev = O.initial_state(g, rho, lmax=2)  # boundary data from the base density: held fixed
        O.run(g, phi, prev, r, T)
        return phi[1:-1, 1:-1, 1:-1]

    def loss(r):
        return float(np.sum(w * (forward(r) - target) ** 2))

    lam = 2 * w * (forward(rho) - target)
    grad = O.adjoint(g, lam, T)
    rng = np.random.default_rng(7)
    for _ in range(6):
        k, j, i = rng.integers(0, g.nz), rng.integers(0, g.ny), rng.integers(0, g.nx)
        eps = 1e-2
        rp = rho.copy()
        rp[k, j, i] += eps
        rm = rho.copy()
        rm[k, j, i] -= eps
        fd = (loss(rp) - loss(rm)) / (2 * eps)
        assert abs(fd - grad[k, j, i]) <= 1e-8 * np.abs(grad).max()


@pytest.mark.parametrize("bc", [O.BC_DIRICHLET, O.BC_ROBIN, O.BC_PERIODIC])
def test_adjoint_dot_product(bc):
    g = _grid(7, 6, 8, 0.1, bc, cfl=0.7)
    T = 30
    drho = I.noise(g.shape, 41, -1.0, 1.0)
    mu = I.noise(g.shape, 42, -1.0, 1.0)
    # linear part of rho -> phi^T: zero initial data and zero boundary data
    phi = O.ghosted(g)
    prev = O.ghosted(g)
    O.run(g, phi, prev, drho, T)
    lhs = np.sum(phi[1:-1, 1:-1, 1:-1] * mu)
    rhs = np.sum(drho * O.adjoint(g, mu, T))
    assert abs(lhs - rhs) < 1e-11 * max(abs(lhs), 1e-30)


def test_periodic_poisson_reference_of_the_lag_study():
    """The lag study's reference (bench.poisson_periodic) solves the discrete periodic Poisson problem exactly."""
    import bench

    n, h = 24, 1.0 / 24
    rho = I.blob_density(n, I.orbit_blobs(0.07))
    phi = bench.poisson_periodic(rho, h)
    lap = sum(np.roll(phi, s, a) for a in range(3) for s in (1, -1)) - 6.0 * phi
    r = lap / h ** 2 - 4.0 * np.pi * (rho - rho.mean())
    assert np.abs(r).max() <= 1e-12 * np.abs(4.0 * np.pi * rho).max()
    assert abs(phi.mean()) < 1e-14


def test_dirichlet_poisson_reference_of_the_domain_study():
    """The domain study's reference (bench.poisson_dirichlet) solves Lap_h phi = 4 pi G rho with the given face
    ghosts exactly, and with the free-space boundary data of a blob it approaches the blob's continuum potential."""
    import bench

    n, h, lo = 20, 1.0 / 20, -0.5
    rng = np.random.Generator(np.random.PCG64(9))
    rho = rng.uniform(0.0, 1.0, (n, n, n))
    ghosts = rng.uniform(-1.0, 0.0, (n + 2, n + 2, n + 2))
    phi = bench.poisson_dirichlet(rho, ghosts, h)
    full = ghosts.copy()
    full[1:-1, 1:-1, 1:-1] = phi
    lap = sum(np.roll(full, s, a) for a in range(3) for s in (1, -1))[1:-1, 1:-1, 1:-1] - 6.0 * phi
    assert np.abs(lap / h ** 2 - 4.0 * np.pi * rho).max() <= 1e-10 * 4.0 * np.pi
    # one Gaussian blob: the discrete solution converges to the continuum potential at second order
    blobs = I.orbit_blobs(0.0)[:1]
    errs = []
    for n in (24, 48):
        h = 1.0 / n
        c = lo + (np.arange(-1, n + 1) + 0.5) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        exact = bench.blob_potential(blobs, X, Y, Z)
        phi = bench.poisson_dirichlet(I.blob_density(n, blobs), exact, h)
        e = exact[1:-1, 1:-1, 1:-1]
        errs.append(np.linalg.norm(phi - e) / np.linalg.norm(e))
    assert errs[1] < 2e-3 and errs[0] / errs[1] > 3.5


def test_exact_sum_is_the_correctly_rounded_sum():
    """The oracle's sums (moments, mass, mean) are the exact sum rounded once; pinned bit for bit against the
    library routine math.fsum (which returns exactly that) on inputs where a running sum goes wrong: massive
    cancellation, a dynamic range beyond 2^1000, exact ties between two doubles (rounded to even, and pushed off
    the tie by a tiny remainder of either sign), and long random sums with a known exact cancellation."""
    import math

    rng = np.random.default_rng(11)
    cases = [
        [],
        [0.0, -0.0],
        [1.0, 1e100, 1.0, -1e100],
        [1e300, 1e300, -1e300, -1e300, 1e-300],
        [1.0, 2.0 ** -53],                      # tie, 1 is even: stays 1
        [1.0 + 2.0 ** -52, 2.0 ** -53],        # tie, rounds up to the even neighbour
        [1.0, 2.0 ** -53, 2.0 ** -200],        # just above the tie: rounds up
        [1.0 + 2.0 ** -52, 2.0 ** -53, -2.0 ** -200],  # just below the tie: rounds down
        [1.0, -2.0 ** -54, -2.0 ** -300],
        [2.0 ** 53, 1.0, 2.0 ** -60, -(2.0 ** 53)],
        [float(v) for v in rng.standard_normal(10000) * 10.0 ** rng.integers(-30, 30, 10000)],
    ]
    big = rng.standard_normal(200000) * 10.0 ** rng.integers(-8, 8, 200000)
    cases.append(list(np.concatenate([big, -big[::-1], [3.5e-17]])))
    cases.append(list(rng.random(100000)))
    for c in cases:
        got = O.exact_sum(np.array(c, dtype=np.float64))
        want = math.fsum(c)
        assert got == want or (got == 0.0 and want == 0.0), (got, want)
    # the running sum of the same random cancellation case is far off; the exact one is not
    a = np.concatenate([big, -big[::-1], [3.5e-17]])
    assert O.exact_sum(a) == 3.5e-17
    g = O.unit_cube(8, 1.0, 1.0, 0.5, O.BC_PERIODIC)
    rho = rng.random((8, 8, 8))
    assert O.mass(g, rho) == math.fsum(rho.ravel()) * g.h * g.h * g.h
    assert O.mean(g, rho) == math.fsum(rho.ravel()) / rho.size


@pytest.mark.parametrize("bc", [O.BC_ROBIN, O.BC_PERIODIC, O.BC_DIRICHLET])
def test_all_core_timing_build_computes_the_same_bits(bc):
    """The benchmark times the oracle on all host cores with an OpenMP build of the same C file; it must compute
    exactly what the checked single-threaded oracle computes."""
    n = 20
    g = O.unit_cube(n, 1.0, 1.0, 0.5, bc, ny=17, nz=23)
    rho = I.blob_density(n, I.draw_blobs(3, 4), 17, 23) + 0.1
    p, q = O.initial_state(g, rho, lmax=2)
    p2, q2 = p.copy(), q.copy()
    O.run(g, p, q, rho, 30)
    O.run_all_cores(g, p2, q2, rho, 30, threads=4)
    assert np.array_equal(p, p2) and np.array_equal(q, q2)
