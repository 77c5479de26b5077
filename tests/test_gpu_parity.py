"""GPU-vs-oracle parity through the C ABI (needs a GB300 and the built library).

Tolerances (after the stated number of sub-steps, over interior cells):
  FP64 path   : relative L-inf <= 1e-12
  FP32-Kahan  : relative L2 <= 1e-5 and relative L-inf <= 1e-4
Shapes are odd and ragged on purpose: 133 x 37 x 29 spans two 128-cell x tiles plus a tail, 4.6 y tiles of 8 rows
and a partial z chunk; 96 x 20 x 17 puts the +x ghost in the first lane past the last cell group; 256 x 9 x 11
fills whole x tiles.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402

BC_PAIRS = {"dirichlet": O.BC_DIRICHLET, "multipole": O.BC_DIRICHLET, "robin": O.BC_ROBIN, "periodic": O.BC_PERIODIC}


@pytest.fixture(scope="module", autouse=True)
def _built():
    hg.build()


def pair(nx, ny, nz, h, bc, prec, lmax=0, c=1.0, G=1.0, cfl=0.5, origin=None):
    origin = origin or (-0.5 * nx * h, -0.5 * ny * h, -0.5 * nz * h)
    dt = cfl * h / (c * np.sqrt(3.0))
    g = hg.Grid(nx, ny, nz, h, origin, c, G, dt, prec, bc, lmax)
    og = O.Grid(nx, ny, nz, h, origin, c, G, dt, BC_PAIRS[bc])
    return g, og


def robin_cfl(nx, ny, nz, h):
    """Largest Courant number (times 0.9) at which every face ghost of a centred box keeps nu / mu <= 1."""
    n = (nx, ny, nz)
    o = [-0.5 * m * h for m in n]
    mu_min = 1.0
    for ax in range(3):
        for side in (0, 1):
            idx = [np.arange(m) for m in n]
            idx[ax] = np.array([-1 if side == 0 else n[ax]])
            X, Y, Z = np.meshgrid(*[o[a] + (idx[a] + 0.5) * h for a in range(3)], indexing="ij")
            r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
            mu_min = min(mu_min, float((np.abs((X, Y, Z)[ax]) / r).min()))
    return min(0.5, 0.9 * np.sqrt(3.0) * mu_min)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def check(prec, a, b, what=""):
    l2, linf = rel(a, b)
    if prec == "f64":
        assert linf <= 1e-12, f"{what} f64 rel Linf {linf:.3e}"
    else:
        assert l2 <= 1e-5 and linf <= 1e-4, f"{what} f32k rel L2 {l2:.3e} Linf {linf:.3e}"
    return l2, linf


@pytest.mark.parametrize("shape", [(133, 37, 29), (96, 20, 17), (256, 9, 11)])
@pytest.mark.parametrize("prec", ["f64", "f32k"])
@pytest.mark.parametrize("bc", ["dirichlet", "multipole", "robin", "periodic"])
def test_seeded_steps_ragged(prec, bc, shape):
    nx, ny, nz = shape
    h = 1.0 / 64
    # Robin needs nu / mu <= 1 on every face: elongated boxes have oblique faces, hence the smaller Courant number
    g, og = pair(nx, ny, nz, h, bc, prec, lmax=3 if bc == "multipole" else 0,
                 cfl=robin_cfl(nx, ny, nz, h) if bc == "robin" else 0.5)
    rho = I.noise(og.shape, 101, 0.0, 2.0)
    phi0 = I.noise(og.shape, 102, -1.0, -0.5)
    prev0 = phi0 + 1e-3 * I.noise(og.shape, 103, -1.0, 1.0)
    g.set_density(torch.from_numpy(rho).cuda())
    g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
    p, q = O.initial_state(og, rho, lmax=g.lmax, phi0=phi0, phi_prev0=prev0)
    # ghosts at t = 0 agree (Dirichlet data / Robin static limit / periodic copies)
    G0 = g.phi_ghosted()
    check(prec, G0, p, "ghosted t=0")
    for n in (1, 6):
        g.step(n)
        O.run(og, p, q, rho, n)
    G1 = g.phi_ghosted()
    check(prec, G1[1:-1, 1:-1, 1:-1], p[1:-1, 1:-1, 1:-1], "interior")
    check(prec, G1, p, "with ghosts")
    assert g.stats()["step"] == 7
    if prec == "f64" and bc == "robin":
        # the FP64 update and the Robin ghost formula round operation by operation like the plain evaluation, so with
        # seeded data (no multipole moments, no mean density) the GPU reproduces the oracle bit for bit
        assert np.array_equal(G1, p)


@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_sphere_dirichlet_analytic_32(prec):
    """Config-1 density (uniform sphere, R = 1/4, 4^3 sub-sampled) with -GM/r boundary data, phi = 0 at t = 0."""
    n = 32
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, prec, "dirichlet")
    og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    rho = I.sphere_density(n)
    g.set_density(rho)
    p, q = O.initial_state(og, rho)
    g.step(600)
    O.run(og, p, q, rho, 600)
    check(prec, g.phi(torch.float64, "cpu"), p[1:-1, 1:-1, 1:-1], "sphere")
    st = g.stats()
    assert abs(st["mass"] - O.mass(og, rho)) < 1e-13
    rms, mx = O.residual(og, p, rho)
    assert abs(st["residual_max"] - mx) < (1e-9 if prec == "f64" else 1e-3) * mx


def test_sphere_robin_run_to_convergence_24():
    """Config 1 with the absorbing boundary, run to convergence on the GPU (the paper's stopping rule: relative change
    per sub-step below 1e-10): the converged FP64 potential is the discrete Robin-Poisson fixed point (sparse direct
    solve) and the analytic sphere within its discretisation error; the compensated-FP32 grid run for the same
    number of sub-steps lands on the same fixed point within its tolerance."""
    from tests import poisson_ref as R
    n = 24
    rho = I.sphere_density(n)
    og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN)
    fixed = R.robin_poisson(og.h, og.G, og.origin, rho)
    X, Y, Z = og.centres()
    an = R.analytic_sphere(X, Y, Z)
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, "f64", "robin")
    g.set_density(rho)
    steps = 0
    while steps < 100000:
        g.step(500)
        steps += 500
        if g.stats()["change_rel"] < 1e-10:
            break
    assert g.stats()["change_rel"] < 1e-10, steps
    u = g.phi(torch.float64, "cpu")
    assert np.abs(u - fixed).max() < 1e-6 * np.abs(fixed).max(), (steps, np.abs(u - fixed).max())
    assert np.sqrt(np.mean((u - an) ** 2) / np.mean(an ** 2)) < 5e-3
    g32 = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, "f32k", "robin")
    g32.set_density(rho)
    g32.step(steps)
    u32 = g32.phi(torch.float64, "cpu")
    assert np.abs(u32 - fixed).max() < 1e-5 * np.abs(fixed).max()


@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_precision_config_2000_substeps(prec):
    """Config-2 workload at 64^3 (the oracle's size): sphere + 8 blobs (seed 1), multipole l <= 4, 2000 sub-steps."""
    n = 64
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, prec, "multipole", lmax=4)
    og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    rho = I.sphere_density(n) + I.blob_density(n, I.draw_blobs(8, 1))
    g.set_density(torch.from_numpy(rho).cuda())
    p, q = O.initial_state(og, rho, lmax=4)
    g.step(2000)
    O.run(og, p, q, rho, 2000)
    check(prec, g.phi(torch.float64, "cpu"), p[1:-1, 1:-1, 1:-1], "config-2 64^3")
    Q = g.moments()
    Qo = O.moments(og, rho, 4)
    assert np.abs(Q - Qo).max() <= 1e-12 * np.abs(Qo).max()


@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_accel_and_compare(prec):
    nx, ny, nz = 70, 45, 33
    g, og = pair(nx, ny, nz, 1.0 / 48, "robin", prec)
    rho = I.blob_density(nx, I.draw_blobs(4, 5), ny, nz, h=og.h, lo=og.origin[0])
    g.set_density(rho)
    p, q = O.initial_state(og, rho)
    g.step(50)
    O.run(og, p, q, rho, 50)
    ax, ay, az = g.accel(torch.float64)
    rx, ry, rz = O.accel(og, p)
    for a, r in ((ax, rx), (ay, ry), (az, rz)):
        l2, linf = rel(a.cpu().numpy(), r)
        assert (linf <= 1e-11) if prec == "f64" else (l2 <= 1e-4)
    ax32, _, _ = g.accel(torch.float32)
    assert np.linalg.norm(ax32.cpu().numpy() - rx) / np.linalg.norm(rx) < 1e-4
    ref = p.copy()
    ref[1:-1, 1:-1, 1:-1] *= 1.001
    got = g.compare(ref[1:-1, 1:-1, 1:-1])
    want = O.compare(og, p, ref)
    # the metrics themselves are FP64 reductions; for f32k they inherit the ~1e-8 relative deviation of phi
    assert np.allclose(got, want, rtol=1e-10, atol=1e-6 if prec == "f32k" else 1e-13)


def test_periodic_mean_removed_and_plane_wave():
    n = 40
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.9, "f64", "periodic")
    X, Y, Z = O.unit_cube(n, 1.0, 1.0, 0.9, O.BC_PERIODIC).centres()
    k = 2 * np.pi * np.array([1, 2, 0])
    nu = g.c * g.dt / g.h
    w = np.arccos(1 - 2 * nu ** 2 * np.sum(np.sin(k * g.h / 2) ** 2))
    kx = k[0] * X + k[1] * Y + k[2] * Z
    g.set_density(np.zeros((n, n, n)))
    g.set_phi(np.cos(kx), np.cos(kx + w))
    g.step(500)
    assert np.abs(g.phi(torch.float64, "cpu") - np.cos(kx - 500 * w)).max() < 1e-10


def test_checkpoint_resume_bit_exact():
    n = 48
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, "f32k", "robin")
    g.set_density(I.sphere_density(n))
    g.step(30)
    blob = g.save_state()
    g.step(25)
    a = g.phi(torch.float64, "cpu")
    g.load_state(blob)
    assert g.stats()["step"] == 30
    g.step(25)
    b = g.phi(torch.float64, "cpu")
    assert np.array_equal(a, b)


def test_load_state_rejects_other_grid_parameters():
    """A checkpoint carries the scaled source, the Dirichlet data and the Robin coefficients of the grid that wrote
    it; a grid of the same shape but another dt, c_h, G, h or origin must refuse it and keep its own state."""
    n = 16
    h = 1.0 / n
    o = (-0.5, -0.5, -0.5)
    dt = 0.5 * h / np.sqrt(3.0)
    g = hg.Grid(n, n, n, h, o, 1.0, 1.0, dt, "f64", "robin")
    g.set_density(I.sphere_density(n))
    g.step(5)
    blob = g.save_state()
    others = [hg.Grid(n, n, n, h, o, 1.0, 1.0, dt * 0.5, "f64", "robin"),
              hg.Grid(n, n, n, h, o, 0.5, 1.0, dt, "f64", "robin"),
              hg.Grid(n, n, n, h, o, 1.0, 2.0, dt, "f64", "robin"),
              hg.Grid(n, n, n, h * 0.5, (-0.25, -0.25, -0.25), 1.0, 1.0, dt * 0.5, "f64", "robin"),
              hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5 + h), 1.0, 1.0, dt, "f64", "robin")]
    for g2 in others:
        g2.set_density(I.sphere_density(n))
        g2.step(2)
        before = g2.phi(torch.float64, "cpu")
        with pytest.raises(hg.HGError):
            g2.load_state(blob)
        assert np.array_equal(g2.phi(torch.float64, "cpu"), before)
        assert g2.stats()["step"] == 2
        g2.free()
    g3 = hg.Grid(n, n, n, h, o, 1.0, 1.0, dt, "f64", "robin")
    g3.load_state(blob)
    assert np.array_equal(g3.phi(torch.float64, "cpu"), g.phi(torch.float64, "cpu"))


def test_errors_reported_not_raised_on_device():
    n = 16
    g = hg.Grid.unit_cube(n, 1.0, 1.0, 0.5, "f32k", "robin")
    rho = np.zeros((n, n, n))
    rho[3, 4, 5] = np.nan
    g.set_density(rho)
    g.step(3)
    st = g.stats(check=False)
    assert st["rc"] == hg._lib.HG_ERR_NONFINITE and st["nonfinite"] == 1
    with pytest.raises(hg.HGError):
        g.stats()
    with pytest.raises(hg.HGError):
        hg.Grid.unit_cube(n, 1.0, 1.0, 1.2, "f64", "robin")  # CFL
    with pytest.raises(hg.HGError):
        hg.Grid(8, 8, 8, 0.1, (0.0, 0.0, 0.0), 1.0, 1.0, 0.01, "f64", "robin")  # origin outside: Robin undefined
    with pytest.raises(hg.HGError):
        g.set_density(np.zeros((n, n, n + 1)))
