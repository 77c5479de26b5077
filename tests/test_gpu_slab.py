"""Slab decomposition along z on the GPU (Sec. 4 timing discussion and Sec. 5: the method needs only neighbour
communication): a grid split into 2 or 3 slabs, each a library grid with z interfaces, exchanging one boundary plane
per interface before every sub-step, must reproduce the whole grid's sub-steps bit for bit (FP64 and compensated FP32,
Robin, and multipole Dirichlet with the summed moments) -- in one process (LocalExchange, device copies) and as two
processes sharing the GPU with the planes staged through host memory over gloo (DistExchange; the processes'
kernels never wait on each other: the exchange happens on the host between sub-steps).  h = 1/64, so the slabs'
cell coordinates round exactly as the whole grid's."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from paper_1602_05700_gb300 import slab as S  # noqa: E402

NX, NY, NZ, STEPS, LMAX = 64, 57, 61, 40, 3
H = 1.0 / 64
ORIGIN = (-0.5, -0.4375, -0.46875)  # on the grid of h = 1/64: every cell coordinate is exact
DT = 0.5 * H / np.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    hg.build()


def density():
    return I.blob_density(NX, I.draw_blobs(4, 31), NY, NZ, h=H, lo=-0.5) + 0.05


def whole(prec, bc, rho, Q=None):
    g = hg.Grid(NX, NY, NZ, H, ORIGIN, 1.0, 1.0, DT, prec, bc, LMAX if bc == "multipole" else 0)
    g.set_density(rho)
    if Q is not None:
        g.set_boundary_moments(Q)
    g.step(STEPS)
    out = g.phi(torch.float64, "cpu")
    g.free()
    return out


def slabs_local(prec, bc, rho, parts):
    slabs = [S.GridSlab(NX, NY, k0, k1, H, ORIGIN, 1.0, 1.0, DT, prec, bc, r, parts,
                        LMAX if bc == "multipole" else 0) for r, (k0, k1) in enumerate(S.split_z(NZ, parts))]
    for s in slabs:
        s.grid.set_density(np.ascontiguousarray(rho[s.k0:s.k1]))
    Q = None
    if bc == "multipole":
        Q = S.sum_moments([s.local_moments() for s in slabs])
        for s in slabs:
            s.set_boundary_moments(Q)
    S.SlabRun(slabs, S.LocalExchange(slabs)).step(STEPS)
    out = np.concatenate([s.grid.phi(torch.float64, "cpu") for s in slabs], axis=0)
    for s in slabs:
        s.grid.free()
    return out, Q


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32k"])
@pytest.mark.parametrize("bc", ["robin", "multipole"])
def test_local_slabs_reproduce_the_whole_grid(parts, prec, bc):
    rho = density()
    got, Q = slabs_local(prec, bc, rho, parts)
    want = whole(prec, bc, rho, Q)
    assert np.array_equal(got, want), np.abs(got - want).max()
    if prec == "f64":  # and the oracle's whole-grid run (its moments are the exact sums)
        og = O.Grid(NX, NY, NZ, H, ORIGIN, 1.0, 1.0, DT, O.BC_ROBIN if bc == "robin" else O.BC_DIRICHLET)
        p, q = O.initial_state(og, rho, lmax=LMAX if bc == "multipole" else 0)
        O.run(og, p, q, rho, STEPS)
        ref = p[1:-1, 1:-1, 1:-1]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_slab_calls_reject_what_they_do_not_support():
    s = S.GridSlab(NX, NY, 0, 20, H, ORIGIN, 1.0, 1.0, DT, "f32k", "robin", 0, 2)
    with pytest.raises(hg.HGError):
        s.grid.set_temporal_depth(2)  # the exchange is per sub-step
    with pytest.raises(hg.HGError):
        s.put_ghost(0, s.plane_buffer())  # the -z face of slab 0 is an outer face, not an interface
    with pytest.raises(hg.HGError):
        hg.Batch([s.grid])
    s.grid.free()
    g = hg.Grid(NX, NY, NZ, H, ORIGIN, 1.0, 1.0, DT, "f64", "periodic")
    with pytest.raises(hg.HGError):
        hg._lib.check(hg._lib.lib().hg_set_z_interface(g.handle, 1, 0))
    g.free()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, prec, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK="0")
    import torch.distributed as dist

    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    k0, k1 = S.split_z(NZ, world)[rank]
    s = S.GridSlab(NX, NY, k0, k1, H, ORIGIN, 1.0, 1.0, DT, prec, "robin", rank, world)
    s.grid.set_density(np.ascontiguousarray(density()[k0:k1]))
    S.SlabRun([s], S.DistExchange(s, host=True)).step(STEPS)
    out.put((rank, s.grid.phi(torch.float64, "cpu")))
    s.grid.free()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_two_processes_with_gloo_reproduce_the_whole_grid(prec):
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, prec, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([r[1] for r in res], axis=0)
    assert np.array_equal(got, whole(prec, "robin", density()))
