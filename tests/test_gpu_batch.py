"""Batched grids (one launch per sub-step for all grids, replayed from a CUDA graph): bit-identical to stepping
each grid alone, for mixed sizes, precisions and boundary conditions, across graph replays, autotuning and grids
stepped on their own in between."""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from tests.test_gpu_parity import check  # noqa: E402

SPECS = [(40, "f32k", "robin"), (33, "f64", "robin"), (64, "f32k", "multipole"), (21, "f64", "periodic"),
         (48, "f32k", "periodic"), (96, "f64", "dirichlet"), (130, "f32k", "robin")]


def make(specs, seed):
    grids = []
    for i, (n, prec, bc) in enumerate(specs):
        g = hg.Grid.unit_cube(n, precision=prec, bc=bc, lmax=3 if bc == "multipole" else 0)
        rho = I.blob_density(n, I.draw_blobs(1 + i % 6, seed + i))
        g.set_density(torch.from_numpy(rho).cuda())
        phi0 = -0.1 - 0.01 * I.noise((n, n, n), seed + 100 + i, 0.0, 1.0)
        g.set_phi(torch.from_numpy(phi0).cuda())
        grids.append(g)
    return grids


def test_batch_equals_individual_steps():
    a = make(SPECS, 70)
    b = make(SPECS, 70)
    batch = hg.Batch(a)
    batch.step(13)       # autotunes on its first sub-steps
    assert batch.info()["z_planes_per_block"] > 0
    batch.step(13)       # replays the graph
    a[1].step(3)         # a grid stepped on its own between batch steps
    batch.step(6)
    for g in b:
        g.step(32)
    b[1].step(3)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.phi_ghosted(), gb.phi_ghosted())
        assert ga.stats()["step"] == gb.stats()["step"]


@pytest.mark.parametrize("subset", ["mixed", "f32k", "f64"])
@pytest.mark.parametrize("split", [False, True])
def test_pinned_launch_modes_equal_individual_steps(split, subset):
    """Both launch modes, pinned (one launch for both precisions, or one per precision class on two streams), for a
    mixed batch and for each class alone: bit-identical to stepping each grid alone, across a mode change."""
    specs = [sp for sp in SPECS if subset == "mixed" or sp[1] == subset]
    a = make(specs, 90)
    b = make(specs, 90)
    batch = hg.Batch(a)
    batch.set_split(split)
    batch.step(9)
    assert batch.info()["precisions_in_separate_launches"] == split
    batch.set_split(not split)  # re-tuned for the other mode on the next step
    batch.step(5)
    assert batch.info()["precisions_in_separate_launches"] == (not split)
    batch.set_split(None)
    batch.step(4)
    for g in b:
        g.step(18)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga.phi_ghosted(), gb.phi_ghosted())
    batch.free()
    with pytest.raises(hg.HGError):
        hg._lib.check(hg._lib.lib().hg_batch_set_split(None, 0))


def test_batch_against_oracle():
    specs = [(24, "f64", "robin"), (20, "f32k", "robin"), (28, "f64", "multipole")]
    grids = make(specs, 80)
    batch = hg.Batch(grids)
    batch.step(40)
    for i, (n, prec, bc) in enumerate(specs):
        og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN if bc == "robin" else O.BC_DIRICHLET)
        rho = I.blob_density(n, I.draw_blobs(1 + i % 6, 80 + i))
        phi0 = -0.1 - 0.01 * I.noise((n, n, n), 80 + 100 + i, 0.0, 1.0)
        p, q = O.initial_state(og, rho, lmax=3 if bc == "multipole" else 0, phi0=phi0)
        O.run(og, p, q, rho, 40)
        check(prec, grids[i].phi(torch.float64, "cpu"), p[1:-1, 1:-1, 1:-1], f"batch grid {i}")


def test_batch_rejects_bad_input():
    g = hg.Grid.unit_cube(16)
    with pytest.raises(hg.HGError):
        hg.Batch([g, g])
    with pytest.raises(hg.HGError):
        hg.Batch([])
