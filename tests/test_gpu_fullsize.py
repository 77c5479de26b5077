"""Parity at the benchmark's full size and launch configurations (512^3, Robin, the orbiting-blob density, the
default z chunks the bench uses, single sweeps and the depth-2 fused kernel the headline step runs): sampled outputs
against the oracle, plus a whole-grid property.

After n sub-steps a cell depends only on the initial state within n cells of it (the stencil reaches one cell per
sub-step), so the oracle computes a sampled output on a (2n+1)^3 sub-grid around it, whose frozen ghost layer holds
the initial values (the oracle's Dirichlet mode): those ghosts would only reach the centre after n+1 sub-steps.
FP64 must agree bit for bit (same operation order); the compensated FP32 path within its tolerances.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_1602_05700_gb300 as hg  # noqa: E402

N = 512
NSUB = 4
SAMPLES = 160


@pytest.fixture(scope="module")
def state():
    W = bench.workload(N)
    rho = I.blob_density_torch(N, I.orbit_blobs(0.0), "cuda", torch.float32)
    phi0 = -0.2 + 0.05 * I.noise((N, N, N), 501, -1.0, 1.0)
    prev0 = phi0 + 1e-4 * I.noise((N, N, N), 502, -1.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(503))
    r = NSUB + 1
    pts = rng.integers(r, N - r, size=(SAMPLES, 3))  # (i, j, k), away from the faces
    return W, rho, phi0, prev0, pts


def run_gpu(W, rho, phi0, prev0, prec, depth=1):
    g = hg.Grid(N, N, N, W["h"], W["origin"], W["c"], W["G"], W["dt"], prec, "robin")
    if depth > 1:
        g.set_temporal_depth(depth)  # the default (not exact) mode, as the bench runs it
    g.set_density(rho if prec == "f32k" else rho.double())
    g.set_phi(phi0, prev0)
    g.step(NSUB)
    out = g.phi(torch.float64, "cpu")
    g.free()
    return out


def oracle_samples(W, rho_host, phi0, prev0, pts):
    r = NSUB + 1
    m = 2 * NSUB + 1
    og = O.Grid(m, m, m, W["h"], (0.0, 0.0, 0.0), W["c"], W["G"], W["dt"], O.BC_DIRICHLET)
    out = np.empty(len(pts))
    for s, (i, j, k) in enumerate(pts):
        sl = (slice(k - r, k + r + 1), slice(j - r, j + r + 1), slice(i - r, i + r + 1))
        p = np.ascontiguousarray(phi0[sl])   # ghosted (m+2)^3 block: the ghosts are the initial values, frozen
        q = np.ascontiguousarray(prev0[sl])
        rb = np.ascontiguousarray(rho_host[k - NSUB:k + NSUB + 1, j - NSUB:j + NSUB + 1, i - NSUB:i + NSUB + 1],
                                  dtype=np.float64)
        O.run(og, p, q, rb, NSUB)
        out[s] = p[r, r, r]
    return out


def test_fp64_full_size_bit_exact_on_samples(state):
    W, rho, phi0, prev0, pts = state
    got = run_gpu(W, rho, phi0, prev0, "f64")
    want = oracle_samples(W, rho.double().cpu().numpy(), phi0, prev0, pts)
    g = got[pts[:, 2], pts[:, 1], pts[:, 0]]
    assert np.array_equal(g, want), f"max |diff| {np.abs(g - want).max():.3e}"


@pytest.mark.parametrize("depth", [1, 2])
def test_f32k_full_size_on_samples_and_against_fp64(state, depth):
    W, rho, phi0, prev0, pts = state
    got = run_gpu(W, rho, phi0, prev0, "f32k", depth)
    want = oracle_samples(W, rho.double().cpu().numpy(), phi0, prev0, pts)
    g = got[pts[:, 2], pts[:, 1], pts[:, 0]]
    l2 = np.linalg.norm(g - want) / np.linalg.norm(want)
    linf = np.abs(g - want).max() / np.abs(want).max()
    assert l2 <= 1e-5 and linf <= 1e-4, (l2, linf)
    # a property of the whole grid: the compensated path stays within its tolerance of the FP64 path everywhere
    ref = run_gpu(W, rho, phi0, prev0, "f64")
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    linf = np.abs(got - ref).max() / np.abs(ref).max()
    assert l2 <= 1e-5 and linf <= 1e-4, (l2, linf)
