"""Degenerate and tiny grids through every kernel path: single cells, one-cell-thick slabs and rods in each axis, a
2^3 box, and rods just longer than one 128-cell tile, for every boundary condition and both precisions, against
the oracle; fused sub-steps against single sweeps on the same shapes; and zero sub-steps."""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from tests.test_gpu_parity import check, pair, robin_cfl  # noqa: E402

SHAPES = [(1, 1, 1), (1, 1, 9), (9, 1, 1), (1, 9, 1), (2, 2, 2), (3, 1, 130), (129, 2, 3), (130, 1, 1)]
H = 1.0 / 64


def seeded(shape, seed):
    nz_ny_nx = shape[::-1]
    rho = I.noise(nz_ny_nx, seed, 0.0, 2.0)
    phi0 = I.noise(nz_ny_nx, seed + 1, -1.0, -0.5)
    prev0 = phi0 + 1e-3 * I.noise(nz_ny_nx, seed + 2, -1.0, 1.0)
    return rho, phi0, prev0


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32k"])
@pytest.mark.parametrize("bc", ["dirichlet", "multipole", "robin", "periodic"])
def test_tiny_and_degenerate_grids_against_oracle(prec, bc, shape):
    nx, ny, nz = shape
    g, og = pair(nx, ny, nz, H, bc, prec, lmax=2 if bc == "multipole" else 0,
                 cfl=robin_cfl(nx, ny, nz, H) if bc == "robin" else 0.5)
    rho, phi0, prev0 = seeded(shape, 701)
    g.set_density(torch.from_numpy(rho).cuda())
    g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
    p, q = O.initial_state(og, rho, lmax=g.lmax, phi0=phi0, phi_prev0=prev0)
    g.step(0)
    assert g.stats()["step"] == 0
    for n in (1, 8):
        g.step(n)
        O.run(og, p, q, rho, n)
    G = g.phi_ghosted()
    check(prec, G[1:-1, 1:-1, 1:-1], p[1:-1, 1:-1, 1:-1], f"{shape} interior")
    check(prec, G, p, f"{shape} with ghosts")
    ax, ay, az = g.accel(dtype=torch.float64)
    want = O.accel(og, p)
    scale = max(np.abs(b).max() for b in want)  # components that vanish by symmetry are compared at this scale
    for a, b in zip((ax, ay, az), want):
        assert np.abs(a.cpu().numpy() - b).max() <= (1e-10 if prec == "f64" else 1e-3) * scale


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", ["dirichlet", "robin", "periodic"])
@pytest.mark.parametrize("depth", [2, 3, 8])
def test_fused_equals_single_sweeps_on_degenerate_grids(depth, bc, shape):
    nx, ny, nz = shape
    rho, phi0, prev0 = seeded(shape, 711)
    out = []
    for d in (1, depth):
        g, _ = pair(nx, ny, nz, H, bc, "f32k", cfl=robin_cfl(nx, ny, nz, H) if bc == "robin" else 0.5)
        if d > 1:
            g.set_temporal_depth(d)
            g.set_temporal_exact(True)
        g.set_density(torch.from_numpy(rho).cuda())
        g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
        g.step(7)
        out.append(g.phi_ghosted())
        g.free()
    assert np.array_equal(out[0], out[1])
