"""How far the precision workload's answer moves when its Dirichlet data move by one unit in the last place.

The workload: 256^3 unit cube, the uniform sphere (R = 1/4) plus 8 Gaussian blobs (seed 1), multipole Dirichlet data
with l <= 4 (Sec. 4, model aD05), 2000 sub-steps from phi = 0 at CFL 0.5.  The oracle alone, run four times:
  base     the moments and ghosts as the oracle computes them;
  q_ulp    every moment moved by one unit in the last place (random direction);
  g_ulp    every face ghost moved by one unit in the last place (random direction);
  slabs    the moments summed over 8 z-slabs separately (each exact) and the 8 partial results then added.
Written to conditioning_precision_256.json: relative L-inf and L2 distance of each variant from base after 1000 and
2000 sub-steps.  This fixes what any implementation whose Dirichlet data differ from the oracle's in the last bits
can reach against the 1e-12 relative L-inf bound.  Takes about 10 minutes on 4 host cores.

    python tests/golden/conditioning_precision_256.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N, LMAX, CHECK = 256, 4, (1000, 2000)


def run(kind):
    import oracle as O
    from paper_1602_05700_gb300 import inputs as I

    og = O.unit_cube(N, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    rho = I.sphere_density(N) + I.blob_density(N, I.draw_blobs(8, 1))
    rng = np.random.default_rng(123)
    Q = O.moments(og, rho, LMAX)
    if kind == "q_ulp":
        Q = np.where(rng.random(Q.shape) < 0.5, np.nextafter(Q, np.inf), np.nextafter(Q, -np.inf))
    if kind == "slabs":
        Q = np.zeros_like(Q)
        s = N // 8
        for b in range(8):
            sub = O.Grid(N, N, s, og.h, (og.origin[0], og.origin[1], og.origin[2] + b * s * og.h), og.c, og.G, og.dt,
                         og.bc)
            Q = Q + O.moments(sub, np.ascontiguousarray(rho[b * s:(b + 1) * s]), LMAX)
    p, q = O.ghosted(og), O.ghosted(og)
    O.fill_multipole_ghosts(og, LMAX, Q, p)
    O.fill_multipole_ghosts(og, LMAX, Q, q)
    if kind == "g_ulp":
        face = np.zeros(p.shape, bool)
        face[[0, -1], 1:-1, 1:-1] = face[1:-1, [0, -1], 1:-1] = face[1:-1, 1:-1, [0, -1]] = True
        moved = np.where(rng.random(p.shape) < 0.5, np.nextafter(p, np.inf), np.nextafter(p, -np.inf))
        p[face] = q[face] = moved[face]
    out, done = {}, 0
    for c in CHECK:
        O.run(og, p, q, rho, c - done)
        done = c
        out[c] = p[1:-1, 1:-1, 1:-1].copy()
    return kind, out


if __name__ == "__main__":
    kinds = ["base", "q_ulp", "g_ulp", "slabs"]
    with mp.get_context("spawn").Pool(4) as pool:
        res = dict(pool.map(run, kinds))
    table = {}
    for k in kinds[1:]:
        for c in CHECK:
            b, a = res["base"][c], res[k][c]
            table[f"{k}@{c}"] = {"rel_linf": float(np.abs(a - b).max() / np.abs(b).max()),
                                 "rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(b))}
    with open(os.path.join(HERE, "conditioning_precision_256.json"), "w") as f:
        json.dump({"workload": f"{N}^3 sphere + 8 blobs (seed 1), multipole l <= {LMAX}, CFL 0.5, from phi = 0",
                   "distance_from_base": table}, f, indent=1)
    print(json.dumps(table, indent=1))
