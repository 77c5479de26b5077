"""The FP64 sweep's integer tiers on the GPU (cell.cuh, lap_int.cuh): the sub-step takes the exact-sum form, the
exact-differences form or the plain FP64 form per cell, and every form must give the oracle's bits.  The fields are
built so that each form is taken, and the borders between them are crossed, inside one grid: smooth fields, steep
Gaussian tails, sign changes, exact zeros next to subnormals and tiny normals, values at and one ulp around powers
of two, and phi^{n-1} near and beyond 2 phi^n.  Robin boundary (its ghosts are FP64 operations of the written order
on both sides), so the comparison is bit for bit, signs of zero included.  The single-grid sweep chooses the form per
lane, the batched launches per warp: both are run."""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from tests.test_gpu_parity import robin_cfl  # noqa: E402

SHAPE = (70, 33, 21)  # nx, ny, nz: a 128-cell tile row with a ragged tail, ragged y and z
H = 1.0 / 64
SEEDS = {"smooth": 11, "steep_tails": 12, "sign_changes": 13, "zeros_and_subnormals": 14, "binade_edges": 15,
         "prev_near_2phi": 16}


def radius(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(*[(np.arange(m) + 0.5 - 0.5 * m) * H for m in (nz, ny, nx)], indexing="ij")
    return np.sqrt(x * x + y * y + z * z)


def fields(kind):
    nz, ny, nx = SHAPE[::-1]
    r = radius(SHAPE)
    rng = np.random.default_rng(SEEDS[kind])
    if kind == "smooth":
        phi = -1.0 / np.sqrt(r * r + 0.01)
        prev = phi * (1.0 + 1e-6 * rng.uniform(-1, 1, phi.shape))
    elif kind == "steep_tails":  # neighbour ratios from ~1 to far beyond 2 (tiers 2 and 3)
        phi = -np.exp(-r * r / (2 * 0.03 ** 2)) - 1e-300
        prev = phi * (1.0 - 1e-3)
    elif kind == "sign_changes":
        phi = rng.uniform(-1, 1, (nz, ny, nx))
        prev = phi + 1e-2 * rng.uniform(-1, 1, phi.shape)
    elif kind == "zeros_and_subnormals":
        phi = np.zeros((nz, ny, nx))
        m = rng.uniform(size=phi.shape)
        phi[m < 0.05] = 5e-324 * rng.integers(1, 50, phi.shape)[m < 0.05]  # subnormals
        phi[(m >= 0.05) & (m < 0.08)] = -1e-300
        phi[(m >= 0.08) & (m < 0.10)] = -0.0
        prev = phi.copy()
        prev[m > 0.95] = -1e-310
    elif kind == "binade_edges":  # -2^k exactly or one ulp either side: neighbours one or more binades apart
        k = rng.integers(-3, 3, (nz, ny, nx))
        phi = -np.ldexp(1.0, k)
        sel = rng.uniform(size=phi.shape)
        phi = np.where(sel < 0.33, np.nextafter(phi, 0.0), np.where(sel < 0.66, np.nextafter(phi, -np.inf), phi))
        prev = phi.copy()
    elif kind == "prev_near_2phi":  # |prev| just below, at and above 2|phi|: 2 phi - prev near zero, or of flipped sign
        phi = -1.0 / np.sqrt(r * r + 0.02)
        f = rng.choice([1.9999999, 2.0, 2.0000001, 1.0], phi.shape)
        prev = phi * f
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(phi), np.ascontiguousarray(prev)


@pytest.mark.parametrize("kind", ["smooth", "steep_tails", "sign_changes", "zeros_and_subnormals", "binade_edges",
                                  "prev_near_2phi"])
@pytest.mark.parametrize("with_source", [False, True])
def test_fp64_tiers_bit_exact(kind, with_source):
    nx, ny, nz = SHAPE
    origin = (-0.5 * nx * H, -0.5 * ny * H, -0.5 * nz * H)
    dt = robin_cfl(nx, ny, nz, H) * H / np.sqrt(3.0)
    g = hg.Grid(nx, ny, nz, H, origin, 1.0, 1.0, dt, "f64", "robin")
    og = O.Grid(nx, ny, nz, H, origin, 1.0, 1.0, dt, O.BC_ROBIN)
    rho = I.noise(og.shape, 77, 0.0, 2.0) if with_source else np.zeros(og.shape)
    phi0, prev0 = fields(kind)
    g.set_density(torch.from_numpy(rho).cuda())
    g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
    p, q = O.initial_state(og, rho, phi0=phi0, phi_prev0=prev0)
    for n in (1, 2, 3):
        g.step(n)
        O.run(og, p, q, rho, n)
        G = g.phi_ghosted()
        same = G.view(np.uint64) == p.view(np.uint64)
        assert same.all(), f"{kind}: {int((~same).sum())} cells differ after {g.stats(check=False)['step']} sub-steps"
    g.free()


@pytest.mark.parametrize("split", [False, True])
def test_fp64_tiers_bit_exact_in_a_batch(split):
    """The same fields as FP64 grids of one batch (forms chosen per warp), in both launch modes."""
    nx, ny, nz = SHAPE
    origin = (-0.5 * nx * H, -0.5 * ny * H, -0.5 * nz * H)
    dt = robin_cfl(nx, ny, nz, H) * H / np.sqrt(3.0)
    grids, refs = [], []
    for i, kind in enumerate(SEEDS):
        g = hg.Grid(nx, ny, nz, H, origin, 1.0, 1.0, dt, "f64", "robin")
        og = O.Grid(nx, ny, nz, H, origin, 1.0, 1.0, dt, O.BC_ROBIN)
        rho = I.noise(og.shape, 78 + i, 0.0, 2.0)
        phi0, prev0 = fields(kind)
        g.set_density(torch.from_numpy(rho).cuda())
        g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
        p, q = O.initial_state(og, rho, phi0=phi0, phi_prev0=prev0)
        O.run(og, p, q, rho, 13)
        grids.append(g)
        refs.append(p)
    b = hg.Batch(grids)
    b.set_split(split)
    b.step(13)  # autotunes on its first sub-steps, then replays the graph
    for kind, g, p in zip(SEEDS, grids, refs):
        G = g.phi_ghosted()
        same = G.view(np.uint64) == p.view(np.uint64)
        assert same.all(), f"{kind}: {int((~same).sum())} cells differ"
    b.free()
    for g in grids:
        g.free()
