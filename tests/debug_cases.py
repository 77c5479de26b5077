"""The runs the HG_DEBUG test repeats in a release process and in a process that loads the checked library
(HG_DEBUG=1): every sub-step kernel family on ragged shapes -- single sweeps in both precisions under the four
boundary conditions, the fused depth-2 kernel (default and exact), the generic fused kernel, a mixed batch and two z
slabs.  Each run ends with hg_get_stats, which reports a pending error word (HG_ERR_BOUNDS in a debug build).

Run as a script: python tests/debug_cases.py OUT.npz writes the arrays of run_cases() to OUT.npz.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SHAPE = (61, 45, 37)  # nx, ny, nz: ragged in every direction
H = 1.0 / 64


def _grid(hg, shape, prec, bc, lmax=0, z_interfaces=0, origin=None, dt_cfl=None):
    nx, ny, nz = shape
    o = origin if origin is not None else (-0.5 * nx * H, -0.5 * ny * H, -0.5 * nz * H)
    cfl = dt_cfl if dt_cfl is not None else (0.3 if bc == "robin" else 0.5)
    return hg.Grid(nx, ny, nz, H, o, 1.0, 1.0, cfl * H / np.sqrt(3.0), prec, bc, lmax, z_interfaces=z_interfaces)


def _fill(g, shape, seed, torch, I):
    nx, ny, nz = shape
    rho = I.noise((nz, ny, nx), seed, 0.0, 2.0)
    phi0 = I.noise((nz, ny, nx), seed + 1, -1.0, -0.5)
    prev0 = phi0 + 1e-3 * I.noise((nz, ny, nx), seed + 2, -1.0, 1.0)
    g.set_density(torch.from_numpy(rho).cuda())
    g.set_phi(torch.from_numpy(phi0).cuda(), torch.from_numpy(prev0).cuda())


def run_cases() -> dict:
    import torch

    import paper_1602_05700_gb300 as hg
    from paper_1602_05700_gb300 import inputs as I
    from paper_1602_05700_gb300 import slab as S

    out = {}
    seed = 300
    for prec in ("f32k", "f64"):
        for bc in ("dirichlet", "multipole", "robin", "periodic"):
            g = _grid(hg, SHAPE, prec, bc, lmax=2 if bc == "multipole" else 0)
            _fill(g, SHAPE, seed, torch, I)
            g.step(7)
            g.stats()
            out[f"sweep_{prec}_{bc}"] = g.phi_ghosted()
            out[f"accel_{prec}_{bc}"] = np.stack([a.cpu().numpy() for a in g.accel(torch.float64)])
            g.free()
            seed += 10
    for depth, exact in ((2, False), (2, True), (3, True)):
        for bc in ("multipole", "robin", "periodic"):
            g = _grid(hg, SHAPE, "f32k", bc, lmax=2 if bc == "multipole" else 0)
            g.set_temporal_depth(depth)
            g.set_temporal_exact(exact)
            _fill(g, SHAPE, seed, torch, I)
            g.step(7)
            g.stats()
            out[f"fused{depth}_{'exact' if exact else 'default'}_{bc}"] = g.phi_ghosted()
            g.free()
            seed += 10
    specs = [((40, 40, 40), "f32k", "robin"), ((33, 29, 35), "f64", "dirichlet"), ((24, 24, 24), "f32k", "periodic"),
             ((37, 50, 21), "f64", "robin")]
    grids = []
    for shape, prec, bc in specs:
        g = _grid(hg, shape, prec, bc)
        _fill(g, shape, seed, torch, I)
        grids.append(g)
        seed += 10
    b = hg.Batch(grids)
    b.step(5)
    b.free()
    for i, g in enumerate(grids):
        g.stats()
        out[f"batch_{i}"] = g.phi_ghosted()
        g.free()
    nx, ny, nz = SHAPE
    origin = (-0.5, -0.4375, -0.46875)
    rho = I.noise((nz, ny, nx), seed, 0.0, 2.0)
    slabs = [S.GridSlab(nx, ny, k0, k1, H, origin, 1.0, 1.0, 0.25 * H / np.sqrt(3.0), "f32k", "robin", r, 2)
             for r, (k0, k1) in enumerate(S.split_z(nz, 2))]
    for s in slabs:
        s.grid.set_density(np.ascontiguousarray(rho[s.k0:s.k1]))
    S.SlabRun(slabs, S.LocalExchange(slabs)).step(5)
    for r, s in enumerate(slabs):
        s.grid.stats()
        out[f"slab_{r}"] = s.grid.phi_ghosted()
        s.grid.free()
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import paper_1602_05700_gb300 as hg

    res = run_cases()
    res["_debug_build"] = np.array([1 if hg.is_debug_build() else 0])
    np.savez(sys.argv[1], **res)
