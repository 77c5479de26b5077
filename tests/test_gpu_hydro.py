"""The hydrodynamics that consumes the gravity (include/hg_hydro.h) against the oracle: FP64 bit for bit (the
library fixes the operation order and is built without contraction), FP32 within tolerance; alone and coupled to
the wave-equation gravity (density handed over, sub-steps, -grad phi, source terms), on grids that span several
32 x 8 columns and z chunks with ragged tails, degenerate grids, the virial sums, and at the benchmark's full size
on sampled cells.
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

GAMMA = 5.0 / 3.0


def pair(shape, dtype, h=None, gamma=GAMMA, rho_floor=0.0, p_floor=0.0):
    nz, ny, nx = shape
    h = h or 1.0 / max(shape)
    H = hg.Hydro(nx, ny, nz, h, gamma, rho_floor, p_floor, dtype=dtype)
    return H, O.HydroGrid(nx, ny, nz, h, gamma, rho_floor, p_floor)


def rel_err(a, b):
    """Per-field max |a - b| / max |b| over the 5 conserved planes (largest of the five)."""
    a = np.asarray(a, dtype=np.float64).reshape(5, -1)
    b = np.asarray(b, dtype=np.float64).reshape(5, -1)
    return max(np.abs(a[q] - b[q]).max() / max(np.abs(b[q]).max(), 1e-300) for q in range(5))


@pytest.mark.parametrize("shape", [(23, 19, 37), (9, 40, 70), (1, 1, 1), (1, 1, 64), (40, 1, 1), (1, 33, 1),
                                   (3, 2, 33)])
def test_fp64_hydro_steps_bit_exact(shape):
    H, hgo = pair(shape, "f64")
    W = I.hydro_noise(shape, 11 + sum(shape))
    H.set_primitive(W)
    U = O.hydro_cons(hgo, W)
    assert np.array_equal(H.state("cpu").numpy(), U)
    for s in range(3):
        smax = O.hydro_max_speed(hgo, U)
        assert H.max_speed() == smax
        dt = 0.3 * hgo.h / smax
        H.step(dt)
        O.hydro_step(hgo, U, dt)
        got = H.state("cpu").numpy()
        assert np.array_equal(got, U), f"step {s}: max |diff| {np.abs(got - U).max():.3e}"


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fp64_shock_tube_bit_exact_along_each_axis(axis):
    shape = [1, 1, 1]
    shape[2 - axis] = 96
    H, hgo = pair(tuple(shape), "f64", gamma=1.4)
    W = I.shock_tube(tuple(shape), axis)
    H.set_primitive(W)
    U = O.hydro_cons(hgo, W)
    for _ in range(20):
        dt = 0.3 * hgo.h / O.hydro_max_speed(hgo, U)
        H.step(dt)
        O.hydro_step(hgo, U, dt)
    assert np.array_equal(H.state("cpu").numpy(), U)


def test_fp64_floors_bit_exact():
    """A near-vacuum region that the floors have to catch (rho and P floors both active)."""
    shape = (12, 20, 45)
    H, hgo = pair(shape, "f64", rho_floor=1e-3, p_floor=1e-4)
    W = I.hydro_noise(shape, 5)
    W[0, :, :, 20:25] = 1e-3
    W[4, :, :, 20:25] = 1e-4
    W[1, :, :, :20] = -1.5   # gas streams away from the thin low-density slab on both sides
    W[1, :, :, 25:] = 1.5
    H.set_primitive(W)
    U = O.hydro_cons(hgo, W)
    for _ in range(4):
        dt = 0.3 * hgo.h / O.hydro_max_speed(hgo, U)
        H.step(dt)
        O.hydro_step(hgo, U, dt)
    assert np.array_equal(H.state("cpu").numpy(), U)
    assert U[0].min() >= 1e-3


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_strong_blast(dtype):
    """A point-like blast (pressure ratio 1e5): FP64 bit-exact with the oracle; FP32 finite, positive, and mass and
    energy conserved to its rounding while the shock is inside the box."""
    shape = (40, 36, 44)
    H, hgo = pair(shape, dtype, gamma=1.4)
    W = np.zeros((5,) + shape)
    W[0], W[4] = 1.0, 1e-5
    W[4, 19:21, 17:19, 21:23] = 1.0
    H.set_primitive(W)
    U = O.hydro_cons(hgo, W)
    tot0 = U.reshape(5, -1).sum(axis=1)
    for _ in range(15):
        dt = 0.3 * hgo.h / O.hydro_max_speed(hgo, U)
        H.step(dt)
        O.hydro_step(hgo, U, dt)
    got = H.state("cpu").numpy().astype(np.float64)
    if dtype == "f64":
        assert np.array_equal(got, U)
    else:
        assert np.isfinite(got).all() and got[0].min() > 0
        tot = got.reshape(5, -1).sum(axis=1)
        assert abs(tot[0] - tot0[0]) < 1e-5 * tot0[0] and abs(tot[4] - tot0[4]) < 1e-4 * tot0[4]


@pytest.mark.parametrize("shape", [(23, 19, 37), (1, 1, 1), (1, 1, 64), (40, 1, 1), (1, 33, 1), (3, 2, 33),
                                   (17, 9, 100)])
def test_fp32_hydro_steps_within_tolerance(shape):
    H, hgo = pair(shape, "f32")
    W = I.hydro_noise(shape, 77)
    H.set_primitive(W)
    U = O.hydro_cons(hgo, W)
    for _ in range(5):
        dt = 0.3 * hgo.h / O.hydro_max_speed(hgo, U)
        H.step(dt)
        O.hydro_step(hgo, U, dt)
    assert rel_err(H.state("cpu").numpy(), U) < 2e-5


def coupled_setup(n, prec, kg=5.0, cfl=0.3, pert=0.0, seed=0):
    """Polytrope (n = 3 index, M = 1, R = 1/3, G = 1) on n^3 cells of [-1/2, 1/2]^3, Robin gravity seeded with the
    exact potential; wave speed c = kg * max(c_s + |v|), sub-step dt_g = cfl h / (c sqrt 3)."""
    h = 1.0 / n
    rho, P, phi, info = I.polytrope(n, pert=pert, seed=seed)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = rho, P
    hgo = O.HydroGrid(n, n, n, h, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"])
    U = O.hydro_cons(hgo, W)
    c = kg * O.hydro_max_speed(hgo, U)
    dtg = cfl * h / (c * np.sqrt(3.0))
    og = O.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, O.BC_ROBIN)
    p, q = O.initial_state(og, rho, phi0=phi, phi_prev0=phi)
    g = hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, prec, "robin")
    g.set_phi(torch.from_numpy(phi).cuda())
    H = hg.Hydro(n, n, n, h, GAMMA, hgo.rho_floor, hgo.p_floor, dtype="f64" if prec == "f64" else "f32")
    H.set_primitive(torch.from_numpy(W).cuda())
    return g, H, og, p, q, hgo, U, dtg, phi


@pytest.mark.parametrize("n", [24, 40])
def test_fp64_coupled_step_bit_exact(n):
    g, H, og, p, q, hgo, U, dtg, phi0 = coupled_setup(n, "f64", pert=0.01, seed=3)
    nsub = 8
    for s in range(3):
        H.step(nsub * dtg, g, nsub)
        O.coupled_step(og, p, q, hgo, U, nsub * dtg, nsub)
        assert np.array_equal(H.state("cpu").numpy(), U), f"hydro state, step {s}"
        assert np.array_equal(g.phi_ghosted(), p), f"potential, step {s}"
    v = H.virial(g)
    w = O.hydro_virial(hgo, U, O.interior(p))
    for key in ("W", "U", "K", "M_bound"):
        assert abs(v[key] - w[key]) <= 1e-12 * abs(w[key]) + 1e-300, key
    assert abs(v["VC"] - w["VC"]) <= 1e-10 * max(abs(w["VC"]), 1e-3)
    assert v["rho_max"] == w["rho_max"]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32k", 1e-4)])
def test_coupled_step_with_multipole_dirichlet_gravity(prec, tol):
    """The coupling with the other outer boundary of the paper (Dirichlet data by the multipole expansion, l <= 4,
    recomputed from each hydro step's density): FP64 to rounding (the moments' sums run in another order), FP32
    compensated within its tolerance."""
    n, lmax, kg, cfl = 32, 4, 5.0, 0.3
    h = 1.0 / n
    rho, P, phi, info = I.polytrope(n, pert=0.01, seed=6)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = rho, P
    W[1] = 0.05  # a bulk drift, so the moments change from step to step
    hgo = O.HydroGrid(n, n, n, h, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"])
    U = O.hydro_cons(hgo, W)
    c = kg * O.hydro_max_speed(hgo, U)
    dtg = cfl * h / (c * np.sqrt(3.0))
    og = O.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, O.BC_DIRICHLET)
    p, q = O.initial_state(og, rho, lmax=lmax, phi0=phi, phi_prev0=phi)
    g = hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, prec, "multipole", lmax)
    g.set_density(torch.from_numpy(rho).cuda())
    g.set_phi(torch.from_numpy(phi).cuda())
    H = hg.Hydro(n, n, n, h, GAMMA, hgo.rho_floor, hgo.p_floor, dtype="f64" if prec == "f64" else "f32")
    H.set_primitive(torch.from_numpy(W).cuda())
    nsub = 8
    for _ in range(3):
        H.step(nsub * dtg, g, nsub)
        O.coupled_step(og, p, q, hgo, U, nsub * dtg, nsub, lmax)
    assert rel_err(H.state("cpu").numpy(), U) < tol
    ph = g.phi_ghosted()
    assert np.abs(ph - p).max() < tol * np.abs(p).max()


def test_fp32_coupled_step_within_tolerance():
    n = 40
    g, H, og, p, q, hgo, U, dtg, phi0 = coupled_setup(n, "f32k", pert=0.01, seed=4)
    nsub = 8
    for _ in range(4):
        H.step(nsub * dtg, g, nsub)
        O.coupled_step(og, p, q, hgo, U, nsub * dtg, nsub)
    assert rel_err(H.state("cpu").numpy(), U) < 1e-4
    ph = g.phi_ghosted()[1:-1, 1:-1, 1:-1]
    assert np.abs(ph - p[1:-1, 1:-1, 1:-1]).max() < 1e-5 * np.abs(p).max()
    v, w = H.virial(g), O.hydro_virial(hgo, U, O.interior(p))
    assert abs(v["W"] - w["W"]) < 1e-5 * abs(w["W"]) and abs(v["VC"] - w["VC"]) < 1e-4


def test_launch_count_and_argument_checks():
    H, _ = pair((8, 8, 8), "f32")
    H.set_primitive(I.hydro_noise((8, 8, 8), 1))
    n0 = H.launches()
    H.step(1e-3)
    assert H.launches() - n0 == 2  # one launch per Runge-Kutta stage
    H.profile(True)
    for _ in range(3):
        H.step(1e-3)
    ms, nl = H.profile_read()
    assert nl == 6 and ms > 0.0
    H.profile(False)
    H.step(1e-3)
    assert H.profile_read() == (0.0, 0)
    with pytest.raises(hg.HGError):
        H.step(0.0)
    with pytest.raises(hg.HGError):
        H.step(1e-3, hg.Grid.unit_cube(9), 1)  # grid size mismatch
    with pytest.raises(hg.HGError):
        H.set_state(np.zeros((5, 8, 8, 8)))  # float64 into a float32 state
    with pytest.raises(hg.HGError):
        H.set_primitive(np.zeros((5, 8, 8, 7)))


def test_mixed_precisions_and_side_stream():
    """An FP64 hydro state coupled to a compensated-FP32 gravity grid (the density handed over and a read back in
    the hydro's precision) stays within the FP32 gravity's tolerance of the all-FP64 pair; and a pair created on a
    side stream gives bit-identical results to the default stream."""
    n, nsub = 24, 6
    out = {}
    for key, prec, stream in (("f64", "f64", None), ("mixed", "f32k", None), ("side", "f64", torch.cuda.Stream())):
        ctx = torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(torch.cuda.current_stream())
        with ctx:
            rho, P, phi, info = I.polytrope(n, pert=0.01, seed=8)
            W = np.zeros((5, n, n, n))
            W[0], W[4] = rho, P
            c, h = 12.0, 1.0 / n
            dtg = 0.3 * h / (c * np.sqrt(3.0))
            g = hg.Grid(n, n, n, h, (-0.5, -0.5, -0.5), c, 1.0, dtg, prec, "robin")
            g.set_phi(torch.from_numpy(phi).cuda())
            H = hg.Hydro(n, n, n, h, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"], dtype="f64")
            H.set_primitive(torch.from_numpy(W).cuda())
            for _ in range(3):
                H.step(nsub * dtg, g, nsub)
            out[key] = H.state("cpu").numpy()
    assert np.array_equal(out["side"], out["f64"])
    assert rel_err(out["mixed"], out["f64"]) < 1e-5


@pytest.mark.parametrize("prec", ["f32k", "f64"])
def test_coupled_checkpoint_resume_bit_exact(prec):
    """Checkpoint of a coupled run (the gravity grid's state and the hydro state), resumed into fresh objects:
    the continuation is bit-identical to the uninterrupted run."""
    n, nsub = 24, 6
    g, H, og, p, q, hgo, U, dtg, phi0 = coupled_setup(n, prec, pert=0.01, seed=12)
    for _ in range(2):
        H.step(nsub * dtg, g, nsub)
    gstate, hstate = g.save_state(), H.state("cpu").clone()
    for _ in range(3):
        H.step(nsub * dtg, g, nsub)
    want_h, want_phi = H.state("cpu").numpy(), g.phi_ghosted()
    g2 = hg.Grid(n, n, n, g.h, g.origin, g.c, g.G, g.dt, prec, "robin")
    g2.load_state(gstate)
    H2 = hg.Hydro(n, n, n, g.h, GAMMA, hgo.rho_floor, hgo.p_floor, dtype="f64" if prec == "f64" else "f32")
    H2.set_state(hstate)
    for _ in range(3):
        H2.step(nsub * dtg, g2, nsub)
    assert np.array_equal(H2.state("cpu").numpy(), want_h)
    assert np.array_equal(g2.phi_ghosted(), want_phi)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_state_round_trip_host_and_device(dtype):
    shape = (5, 6, 7)
    H, hgo = pair(shape, dtype)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    U = torch.from_numpy(O.hydro_cons(hgo, I.hydro_noise(shape, 3))).to(tdt)
    H.set_state(U.numpy())                 # from host
    assert torch.equal(H.state("cpu"), U)
    H.set_state((2 * U).cuda())            # from device
    assert torch.equal(H.state("cuda").cpu(), 2 * U)
    with pytest.raises(hg.HGError):
        H.virial(hg.Grid.unit_cube(8))     # grid size mismatch


def test_full_size_sampled_cells_bit_exact():
    """280^3 polytrope (the virial workload's grid) with 1% density perturbations, one FP64 hydro step in the
    launch configuration of the benchmark; 40 sampled cells against the oracle on the 9^3 neighbourhood each
    depends on (two stages, each reaching 2 cells)."""
    n = 280
    rho, P, phi, info = I.polytrope(n, pert=0.01, seed=9)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = rho, P
    W[1:4] = 0.05 * I.noise((3, n, n, n), 10, -1.0, 1.0)
    H = hg.Hydro(n, n, n, 1.0 / n, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"], dtype="f64")
    H.set_primitive(torch.from_numpy(W).cuda())
    dt = 0.3 / n / 3.0  # below the CFL limit: max(c_s + |v|) < 2.3 for this star
    H.step(dt)
    got = H.state("cpu").numpy()
    rng = np.random.Generator(np.random.PCG64(12))
    pts = rng.integers(4, n - 4, size=(40, 3))
    pts[:10] = rng.integers(n // 2 - 60, n // 2 + 60, size=(10, 3))  # inside the star
    sub = O.HydroGrid(9, 9, 9, 1.0 / n, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"])
    for (i, j, k) in pts:
        Wl = np.ascontiguousarray(W[:, k - 4:k + 5, j - 4:j + 5, i - 4:i + 5])
        Ul = O.hydro_cons(sub, Wl)
        O.hydro_step(sub, Ul, dt)
        assert np.array_equal(got[:, k, j, i], Ul[:, 4, 4, 4]), (i, j, k)
    assert H.max_speed() < 3.0
    # the FP32 state (the benchmark's precision) stays within tolerance of the FP64 one over the whole grid
    H.free()
    H32 = hg.Hydro(n, n, n, 1.0 / n, GAMMA, 0.5 * info["rho_atm"], 0.5 * info["p_atm"], dtype="f32")
    H32.set_primitive(torch.from_numpy(W).cuda())
    H32.step(dt)
    assert rel_err(H32.state("cpu").numpy(), got) < 1e-5
