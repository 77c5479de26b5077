"""Temporal blocking (K fused sub-steps per pass) against K single sweeps and against the oracle.

The fused kernels use the same per-cell arithmetic as the single sweep.  In exact mode (hg_set_temporal_exact) their
inner levels also round the compensation as a store would, so the results must be identical bit for bit, for every
boundary condition, for step counts that are not multiples of K, and on ragged shapes whose tiles straddle every
face.  In the default mode the inner levels keep the compensation as a float: the results may differ from single
sweeps only in the compensation's last bits (below 1e-9 of phi), and meet the oracle tolerances.
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
from tests.test_gpu_parity import BC_PAIRS, check, robin_cfl  # noqa: E402


def make(shape, bc, h=1.0 / 64, depth=1, lmax=0, exact=True):
    nx, ny, nz = shape
    origin = (-0.5 * nx * h, -0.5 * ny * h, -0.5 * nz * h)
    cfl = robin_cfl(nx, ny, nz, h) if bc == "robin" else 0.5
    dt = cfl * h / np.sqrt(3.0)
    g = hg.Grid(nx, ny, nz, h, origin, 1.0, 1.0, dt, "f32k", bc, lmax)
    if depth > 1:
        g.set_temporal_depth(depth)
        g.set_temporal_exact(exact)
    og = O.Grid(nx, ny, nz, h, origin, 1.0, 1.0, dt, BC_PAIRS[bc])
    return g, og


@pytest.mark.parametrize("shape", [(61, 45, 37), (96, 31, 70), (30, 30, 30)])
@pytest.mark.parametrize("bc", ["dirichlet", "multipole", "robin", "periodic"])
@pytest.mark.parametrize("depth", [2, 3, 4, 5, 6, 7, 8])
def test_fused_equals_single_sweeps_bitwise(depth, bc, shape):
    rho = I.noise(shape[::-1], 201, 0.0, 2.0)
    phi0 = I.noise(shape[::-1], 202, -1.0, -0.5)
    prev0 = phi0 + 1e-3 * I.noise(shape[::-1], 203, -1.0, 1.0)
    out = []
    for d in (1, depth):
        g, _ = make(shape, bc, depth=d, lmax=2 if bc == "multipole" else 0)
        g.set_density(torch.from_numpy(rho).cuda())
        g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
        g.step(11)  # not a multiple of the depth
        g.step(depth + 1)
        out.append((g.phi_ghosted(), g.stats()))
        g.free()
    a, b = out[0][0], out[1][0]
    assert np.array_equal(a, b), f"max diff {np.abs(a - b).max():.3e}"
    assert out[0][1]["step"] == out[1][1]["step"] == 11 + depth + 1
    assert out[0][1]["change_rel"] == out[1][1]["change_rel"]  # the dlt buffers agree too


@pytest.mark.parametrize("shape", [(61, 45, 37), (96, 31, 70), (128, 17, 40)])
@pytest.mark.parametrize("bc", ["dirichlet", "robin", "periodic"])
@pytest.mark.parametrize("depth", [2, 3])
def test_fused_default_mode_against_single_sweeps_and_oracle(depth, bc, shape):
    """Default mode: the inner levels keep their compensation as a float instead of the stored 16-bit code, so
    roundings of the increment flip here and there (these seeded fields have increments near 0.2, whose unit in the
    last place is 1.5e-8): the result stays within a few of those units of single sweeps, and is at least as close
    to the FP64 oracle as the single sweeps are."""
    rho = I.noise(shape[::-1], 211, 0.0, 2.0)
    phi0 = I.noise(shape[::-1], 212, -1.0, -0.5)
    prev0 = phi0 + 1e-3 * I.noise(shape[::-1], 213, -1.0, 1.0)
    out = []
    for d in (1, depth):
        g, og = make(shape, bc, depth=d, exact=False)
        g.set_density(torch.from_numpy(rho).cuda())
        g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())
        g.step(11)
        g.step(depth + 1)
        out.append(g.phi(torch.float64, "cpu"))
        g.free()
    single, fused = out
    p, q = O.initial_state(og, rho, phi0=phi0, phi_prev0=prev0)
    O.run(og, p, q, rho, 11 + depth + 1)
    ref = p[1:-1, 1:-1, 1:-1]
    assert np.abs(single - fused).max() <= 1e-6 * np.abs(ref).max()
    e_single = np.linalg.norm(single - ref) / np.linalg.norm(ref)
    e_fused = np.linalg.norm(fused - ref) / np.linalg.norm(ref)
    assert e_fused <= 1.05 * e_single + 1e-12, (e_fused, e_single)


@pytest.mark.parametrize("exact", [True, False])
@pytest.mark.parametrize("depth", [2, 4])
def test_fused_against_oracle_sphere_robin(depth, exact):
    n = 48
    g, og = make((n, n, n), "robin", h=1.0 / n, depth=depth, exact=exact)
    rho = I.sphere_density(n)
    g.set_density(rho)
    p, q = O.initial_state(og, rho)
    g.step(400)
    O.run(og, p, q, rho, 400)
    check("f32k", g.phi(torch.float64, "cpu"), p[1:-1, 1:-1, 1:-1], "temporal sphere")


def test_depth_rejected_for_f64_and_out_of_range():
    g = hg.Grid.unit_cube(16, precision="f64", bc="robin")
    with pytest.raises(hg.HGError):
        g.set_temporal_depth(2)
    g2 = hg.Grid.unit_cube(16, precision="f32k", bc="robin")
    with pytest.raises(hg.HGError):
        g2.set_temporal_depth(hg.HG_MAX_TEMPORAL_DEPTH + 1)
    with pytest.raises(hg.HGError):
        g2.set_temporal_depth(0)
