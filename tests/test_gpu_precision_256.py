"""The precision workload at its stated size: a 256^3 grid on the unit cube, the uniform sphere (R = 1/4) plus 8
Gaussian blobs (seed 1), multipole Dirichlet boundary with l <= 4 (Sec. 4, model aD05), 2000 sub-steps from phi = 0,
FP64 and compensated FP32 -- compared element by element with the CPU oracle run on the same input.

Bounds: FP64 relative L-inf <= 1e-12; compensated FP32 relative L2 <= 1e-5 and relative L-inf <= 1e-4.
The oracle's 2000 sub-steps at 256^3 take a few minutes on one host core; they run once per module.
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

N, STEPS, LMAX = 256, 2000, 4


@pytest.fixture(scope="module")
def oracle_run():
    hg.build()
    og = O.unit_cube(N, 1.0, 1.0, 0.5, O.BC_DIRICHLET)
    rho = I.sphere_density(N) + I.blob_density(N, I.draw_blobs(8, 1))
    p, q = O.initial_state(og, rho, lmax=LMAX)
    O.run(og, p, q, rho, STEPS)
    return rho, O.moments(og, rho, LMAX), p[1:-1, 1:-1, 1:-1].copy()


def run_gpu(rho, prec):
    g = hg.Grid.unit_cube(N, 1.0, 1.0, 0.5, prec, "multipole", lmax=LMAX)
    g.set_density(torch.from_numpy(rho).cuda())
    Q = g.moments()
    g.step(STEPS)
    phi = g.phi(torch.float64, "cpu")
    g.free()
    return Q, phi


def test_fp64_config_256_2000_substeps(oracle_run):
    rho, Qo, ref = oracle_run
    Q, phi = run_gpu(rho, "f64")
    # the moments: double-double sums on the GPU against the oracle's exact sums (their terms differ only by the
    # rounding of the harmonics), to a few units in the last place of the largest moment
    assert np.abs(Q - Qo).max() <= 1e-15 * np.abs(Qo).max(), np.abs(Q - Qo).max() / np.abs(Qo).max()
    linf = np.abs(phi - ref).max() / np.abs(ref).max()
    l2 = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    print(f"FP64 256^3 multipole l<=4, {STEPS} sub-steps: rel L-inf {linf:.3e}, rel L2 {l2:.3e}")
    assert linf <= 1e-12, (linf, l2)


def test_f32k_config_256_2000_substeps(oracle_run):
    rho, _, ref = oracle_run
    _, phi = run_gpu(rho, "f32k")
    l2 = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    linf = np.abs(phi - ref).max() / np.abs(ref).max()
    print(f"compensated FP32 256^3 multipole l<=4, {STEPS} sub-steps: rel L2 {l2:.3e}, rel L-inf {linf:.3e}")
    assert l2 <= 1e-5 and linf <= 1e-4, (l2, linf)
