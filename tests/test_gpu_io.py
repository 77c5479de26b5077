"""The pipelined host I/O step (hg_io_step / hg_io_wait) and the sync-free density upload: results bit-identical
to the synchronous calls (set_density, step, accel, copy back) for every precision and boundary condition, the
mass read back lazily, and the argument checks."""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402

CASES = [(40, "f32k", "robin", np.float32), (33, "f64", "robin", np.float64), (36, "f32k", "periodic", np.float64),
         (28, "f64", "multipole", np.float32), (45, "f32k", "dirichlet", np.float32)]


def densities(n, k, seed, dtype):
    return [I.blob_density(n, I.draw_blobs(2 + s % 3, seed + s)).astype(dtype) for s in range(k)]


@pytest.mark.parametrize("keep", [1, 2])
@pytest.mark.parametrize("n,prec,bc,dt", CASES)
def test_io_step_equals_synchronous_calls(n, prec, bc, dt, keep):
    lmax = 3 if bc == "multipole" else 0
    a = hg.Grid.unit_cube(n, precision=prec, bc=bc, lmax=lmax)
    b = hg.Grid.unit_cube(n, precision=prec, bc=bc, lmax=lmax)
    rhos = densities(n, 6, 300 + n, dt)
    adt = np.float64 if prec == "f64" else np.float32
    sets = keep + 1  # output buffer sets in rotation: `keep` calls in flight plus the one checked
    outs = [[np.empty((n, n, n), adt) for _ in range(3)] for _ in range(sets)]
    want = []
    for s, rho in enumerate(rhos):
        a.io_step(rho, 7, outs[s % sets])
        a.io_wait(keep)
        if s >= keep:  # step s - keep is complete: check its output now, before its buffers are reused
            for x, y in zip(outs[(s - keep) % sets], want[s - keep]):
                assert np.array_equal(x, y), f"step {s - keep}"
        b.set_density(torch.from_numpy(rho).cuda())
        b.step(7)
        want.append([t.cpu().numpy() for t in b.accel(dtype=torch.float64 if prec == "f64" else torch.float32)])
    a.io_wait(0)
    for s in range(len(rhos) - keep, len(rhos)):
        for x, y in zip(outs[s % sets], want[s]):
            assert np.array_equal(x, y)
    assert np.array_equal(a.phi_ghosted(), b.phi_ghosted())
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 7 * len(rhos)
    assert sa["mass"] == sb["mass"]


def test_io_step_in_the_bench_configuration():
    """The end-to-end step as the benchmark times it: the orbiting-blob densities at 256^3, Robin, temporal depth 2
    (default mode), 20 sub-steps per call, three calls in flight, page-locked host buffers; every output equals the
    synchronous device-resident step's."""
    import bench

    n, steps, sets = 256, 5, 4
    W = bench.workload(n)
    a = hg.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], "f32k", "robin")
    b = hg.Grid(n, n, n, W["h"], W["origin"], W["c"], W["G"], W["dt"], "f32k", "robin")
    a.set_temporal_depth(2)
    b.set_temporal_depth(2)
    rhos = [I.blob_density_torch(n, I.orbit_blobs(s * W["dt_hyd"]), "cuda", torch.float32) for s in range(steps)]
    host_rho = [r.cpu().pin_memory() for r in rhos]
    outs = [[torch.empty((n, n, n)).pin_memory() for _ in range(3)] for _ in range(sets)]
    want = []
    for s in range(steps):
        a.io_step(host_rho[s], 20, outs[s % sets])
        a.io_wait(sets - 1)
        b.set_density(rhos[s])
        b.step(20)
        want.append([t.cpu() for t in b.accel()])
    a.io_wait(0)
    for s in range(steps - sets + 1, steps):  # the buffers of the last calls still hold their outputs
        for x, y in zip(outs[s % sets], want[s]):
            assert torch.equal(x, y), f"step {s}"
    assert np.array_equal(a.phi_ghosted(), b.phi_ghosted())
    a.free()
    b.free()


def test_io_step_without_density_or_output():
    n = 32
    a = hg.Grid.unit_cube(n)
    b = hg.Grid.unit_cube(n)
    rho = densities(n, 1, 7, np.float32)[0]
    out = [torch.empty((n, n, n), dtype=torch.float32).pin_memory() for _ in range(3)]
    a.io_step(rho, 5)          # density in, no output
    a.io_step(None, 6, out)    # source unchanged, output only
    a.io_step(None, 4)         # neither
    a.io_wait(0)
    b.set_density(torch.from_numpy(rho).cuda())
    b.step(11)
    ref = b.accel()
    b.step(4)
    for x, y in zip(out, ref):
        assert torch.equal(x, y.cpu())
    assert np.array_equal(a.phi_ghosted(), b.phi_ghosted())


@pytest.mark.parametrize("bc", ["robin", "periodic"])
def test_device_density_mass_read_lazily(bc):
    n = 24
    g = hg.Grid.unit_cube(n, precision="f64", bc=bc)
    og = O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_ROBIN if bc == "robin" else O.BC_PERIODIC)
    for s in range(3):
        rho = densities(n, 1, 40 + s, np.float64)[0]
        t = torch.from_numpy(rho).cuda()
        g.set_density(t)
        t.zero_()  # same stream: runs after the source preparation has read it
        g.step(3)
        assert abs(g.stats()["mass"] - O.mass(og, rho)) < 1e-13


def test_density_buffer_reuse_is_stream_ordered():
    n = 40
    a = hg.Grid.unit_cube(n, bc="periodic")
    b = hg.Grid.unit_cube(n, bc="periodic")
    r1, r2 = densities(n, 2, 90, np.float32)
    t = torch.from_numpy(r1).cuda()
    a.set_density(t)
    t.copy_(torch.from_numpy(r2).cuda())  # overwritten right after the call returns
    a.step(9)
    b.set_density(torch.from_numpy(r1).cuda())
    b.step(9)
    assert np.array_equal(a.phi_ghosted(), b.phi_ghosted())


def test_io_step_rejects_bad_input():
    n = 16
    g = hg.Grid.unit_cube(n)
    rho = np.zeros((n, n, n), np.float32)
    with pytest.raises(hg.HGError):
        g.io_step(torch.zeros((n, n, n), device="cuda"), 1)
    with pytest.raises(hg.HGError):
        g.io_step(rho, 1, [np.empty((n, n, n), np.float32)] * 2)
    with pytest.raises(hg.HGError):
        g.io_step(rho, 1, [np.empty((n, n, n), np.float32), np.empty((n, n, n), np.float32),
                           np.empty((n, n, n), np.float64)])
    with pytest.raises(hg.HGError):
        g.io_step(rho, 1, [np.empty((n, n, n + 1), np.float32)] * 3)
    with pytest.raises(hg.HGError):
        g.io_wait(-1)
    g.io_step(rho, 2, [np.empty((n, n, n), np.float32) for _ in range(3)])
    g.io_wait(0)
    assert g.stats()["step"] == 2


def test_bounded_wait_gives_up_and_is_reported():
    """A kernel wait that nothing will satisfy ends after its limit; the host sees the timeout and the grid stays
    usable (no fault, no hang)."""
    import time
    g = hg.Grid.unit_cube(24)
    g.set_density(torch.ones((24, 24, 24), device="cuda"))
    t0 = time.perf_counter()
    g.check_bounded_wait()
    assert time.perf_counter() - t0 < 5.0
    g.step(4)  # the context and the grid still work, and no error is left pending
    g.sync()
    assert g.stats()["step"] == 4
