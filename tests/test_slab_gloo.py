"""Slab decomposition along z (Sec. 4 timing discussion and Sec. 5: only neighbour communication is needed), its
exchange logic on CPU: two and three gloo ranks, each advancing its slab of the oracle's grid and swapping boundary
planes with its neighbours before every sub-step through paper_1602_05700_gb300.slab.DistExchange.  The gathered
slabs must equal the oracle's whole-grid run bit for bit (Robin and multipole Dirichlet; h = 1/32 so that the slabs'
cell coordinates round exactly as the whole grid's)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

N, NZ, STEPS, LMAX = 32, 29, 24, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(bc):
    import oracle as O
    from paper_1602_05700_gb300 import inputs as I

    h = 1.0 / N
    full = O.Grid(N, N - 3, NZ, h, (-0.5, -0.5, -0.5), 1.0, 1.0, 0.5 * h / np.sqrt(3.0), bc)
    rho = I.blob_density(N, I.draw_blobs(3, 21), N - 3, NZ, h=h, lo=-0.5)
    return O, full, rho


class OracleSlab:
    """The oracle's grid restricted to planes k0..k1-1, with the engine calls of slab.GridSlab."""

    def __init__(self, O, full, rho, k0, k1, Q):
        self.O = O
        self.g = O.Grid(full.nx, full.ny, k1 - k0, full.h, (full.origin[0], full.origin[1], full.origin[2] + k0 * full.h),
                        full.c, full.G, full.dt, full.bc)
        self.rho = np.ascontiguousarray(rho[k0:k1])
        self.p, self.q = O.ghosted(self.g), O.ghosted(self.g)
        if full.bc == O.BC_DIRICHLET:  # the whole density's expansion on the slab's faces
            O.fill_multipole_ghosts(self.g, LMAX, Q, self.p)
            O.fill_multipole_ghosts(self.g, LMAX, Q, self.q)

    def plane_buffer(self, device=None):
        return torch.empty((self.g.ny, self.g.nx), dtype=torch.float64)

    def get_plane(self, which, buf):
        buf.copy_(torch.from_numpy(self.p[1 if which == 0 else self.g.nz, 1:-1, 1:-1]))

    def put_ghost(self, side, buf):
        self.p[0 if side == 0 else self.g.nz + 1, 1:-1, 1:-1] = buf.numpy()

    def step_one(self):
        self.O.run(self.g, self.p, self.q, self.rho, 1)


def _worker(rank, world, port, bc, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_1602_05700_gb300 import slab as S

    dist.init_process_group("gloo")
    O, full, rho = _setup(bc)
    k0, k1 = S.split_z(NZ, world)[rank]
    Q = S.sum_moments(O.moments(O.Grid(full.nx, full.ny, k1 - k0, full.h,
                                       (full.origin[0], full.origin[1], full.origin[2] + k0 * full.h), full.c,
                                       full.G, full.dt, full.bc), np.ascontiguousarray(rho[k0:k1]), LMAX),
                      dist_group=True) if bc == O.BC_DIRICHLET else None
    s = OracleSlab(O, full, rho, k0, k1, Q)
    S.SlabRun([s], S.DistExchange(s, host=True)).step(STEPS)
    out.put((rank, k0, s.p[1:-1, 1:-1, 1:-1].copy(), Q))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("bc_name", ["robin", "multipole"])
def test_gloo_slabs_reproduce_the_whole_grid(world, bc_name):
    import oracle as O
    from paper_1602_05700_gb300 import slab as S

    bc = O.BC_ROBIN if bc_name == "robin" else O.BC_DIRICHLET
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bc, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, full, rho = _setup(bc)
    if bc == O.BC_DIRICHLET:
        # the moments of the whole density, added slab by slab, as every rank used them
        Q = res[0][3]
        assert all(np.array_equal(r[3], Q) for r in res)
        assert np.allclose(Q, O.moments(full, rho, LMAX), rtol=0, atol=1e-15 * np.abs(Q).max())
        p, pp = O.ghosted(full), O.ghosted(full)
        O.fill_multipole_ghosts(full, LMAX, Q, p)
        O.fill_multipole_ghosts(full, LMAX, Q, pp)
    else:
        p, pp = O.initial_state(full, rho)
    O.run(full, p, pp, rho, STEPS)
    got = np.concatenate([r[2] for r in res], axis=0)
    assert [r[1] for r in res] == [k0 for k0, _ in S.split_z(NZ, world)]
    assert np.array_equal(got, p[1:-1, 1:-1, 1:-1])


def test_split_z_covers_every_plane_once():
    from paper_1602_05700_gb300 import slab as S

    for nz in (1, 7, 29, 512):
        for parts in range(1, min(nz, 9) + 1):
            r = S.split_z(nz, parts)
            assert r[0][0] == 0 and r[-1][1] == nz and all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [k1 - k0 for k0, k1 in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        S.split_z(3, 4)
