"""Slab decomposition of one grid along z (arXiv 1602.05700, Sec. 4 timing discussion and Sec. 5: the method needs
only communication between neighbouring cells, which suits distributed memory).

The whole grid's nz planes are split into consecutive ranges, each an hg_grid of its own (a "slab", origin shifted
along z).  A sub-step of the whole grid is: every slab's interface ghost planes receive the neighbouring slabs'
boundary planes of phi^n, then every slab advances one sub-step.  The sub-step only reads phi^n one cell away, so
the slabs reproduce the whole grid bit for bit when their cell coordinates (origin + (k + 1/2) h, which set the
boundary data and the Robin coefficients) round as the whole grid's do -- always when h is a power of two and the
origin lies on its grid -- and to rounding otherwise; multipole Dirichlet data also carry the rounding of the
summed moments.

Two independent pieces:
  * an engine per slab with four calls -- plane_buffer(), get_plane(which, buf), put_ghost(side, buf),
    step_one() -- here GridSlab over the library's Grid (the tests also drive the CPU oracle through the same calls);
  * an exchange that moves the planes: LocalExchange (all slabs in this process, copies on the device) or
    DistExchange (one slab per rank, torch.distributed point-to-point: NCCL with device buffers, gloo with host
    buffers).

Interface planes are exchanged before every sub-step (temporal depth 1); the outer faces keep the grid's boundary
condition (Robin, or Dirichlet with the moments of the whole density, see sum_moments).  Periodic grids are not
split (their source needs the mean density of the whole grid).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def split_z(nz: int, parts: int):
    """Consecutive plane ranges [(k0, k1), ...] of nearly equal size covering 0..nz."""
    if parts < 1 or parts > nz:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs")
    base, extra = divmod(nz, parts)
    out, k = [], 0
    for r in range(parts):
        m = base + (1 if r < extra else 0)
        out.append((k, k + m))
        k += m
    return out


class GridSlab:
    """Planes k0..k1-1 of a grid of nz planes (lower corner `origin`), as a library Grid with z interfaces towards
    its neighbours (slab index `index` of `parts`)."""

    def __init__(self, nx, ny, k0, k1, h, origin, c, G, dt, precision, bc, index, parts, lmax=0, stream=None):
        from . import Grid

        self.k0, self.k1, self.index, self.parts = int(k0), int(k1), int(index), int(parts)
        o = (float(origin[0]), float(origin[1]), float(origin[2]) + self.k0 * float(h))
        self.lo, self.hi = self.index > 0, self.index < self.parts - 1
        self.grid = Grid(nx, ny, self.k1 - self.k0, h, o, c, G, dt, precision, bc, lmax, stream,
                         z_interfaces=(1 if self.lo else 0) | (2 if self.hi else 0))
        self.nbytes = int(_lib.lib().hg_plane_bytes(self.grid.handle))

    def plane_buffer(self, device=None):
        import torch

        return torch.empty(self.nbytes, dtype=torch.uint8, device=device if device is not None else self.grid.device)

    def get_plane(self, which: int, buf) -> None:
        _lib.check(_lib.lib().hg_get_plane(self.grid.handle, int(which), ctypes.c_void_p(buf.data_ptr()),
                                           int(buf.is_cuda)))

    def put_ghost(self, side: int, buf) -> None:
        _lib.check(_lib.lib().hg_put_ghost_plane(self.grid.handle, int(side), ctypes.c_void_p(buf.data_ptr()),
                                                 int(buf.is_cuda)))

    def step_one(self) -> None:
        self.grid.step(1)

    def local_moments(self) -> np.ndarray:
        return self.grid.moments()

    def set_boundary_moments(self, Q) -> None:
        self.grid.set_boundary_moments(Q)


class LocalExchange:
    """All slabs in this process: slab r's last plane -> slab r+1's -z ghost, slab r+1's first plane -> slab r's +z
    ghost, through one buffer per interface and direction (device buffers for library slabs)."""

    def __init__(self, slabs):
        self.slabs = list(slabs)
        self.bufs = [(a.plane_buffer(), b.plane_buffer()) for a, b in zip(self.slabs, self.slabs[1:])]

    def exchange(self) -> None:
        for (a, b), (up, down) in zip(zip(self.slabs, self.slabs[1:]), self.bufs):
            a.get_plane(1, up)
            b.get_plane(0, down)
            b.put_ghost(0, up)
            a.put_ghost(1, down)


class DistExchange:
    """One slab per rank of the default process group, rank r holding slab r: the boundary planes go to the ranks
    r-1 and r+1 and their planes come back into the ghost planes, by batched point-to-point operations (no rank
    waits on a send before posting its receives).  host=True stages the planes through host memory (gloo)."""

    def __init__(self, slab, host: bool = False):
        import torch.distributed as dist

        self.slab = slab
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        dev = "cpu" if host else None
        self.send = {s: slab.plane_buffer(dev) for s in (0, 1)}
        self.recv = {s: slab.plane_buffer(dev) for s in (0, 1)}

    def exchange(self) -> None:
        import torch.distributed as dist

        ops, sides = [], []
        if self.rank > 0:
            sides.append((0, self.rank - 1))
        if self.rank < self.world - 1:
            sides.append((1, self.rank + 1))
        for side, peer in sides:
            self.slab.get_plane(side, self.send[side])
        for side, peer in sides:
            ops.append(dist.P2POp(dist.isend, self.send[side], peer))
            ops.append(dist.P2POp(dist.irecv, self.recv[side], peer))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for side, _ in sides:
            self.slab.put_ghost(side, self.recv[side])


class SlabRun:
    """k sub-steps of the whole grid: before each, the exchange fills every interface ghost plane of phi^n, then
    every local slab advances one sub-step."""

    def __init__(self, slabs, exchange):
        self.slabs = list(slabs)
        self.exchange = exchange

    def step(self, n: int) -> None:
        for _ in range(int(n)):
            self.exchange.exchange()
            for s in self.slabs:
                s.step_one()


def sum_moments(local_moments, dist_group: bool = False) -> np.ndarray:
    """The moments of the whole density from the slabs' own moments, added in slab order (the same bits on every
    rank).  local_moments: the list of this process's slabs' moments (LocalExchange), or this rank's one array
    (dist_group=True: gathered over the default process group first)."""
    if not dist_group:
        total = np.zeros_like(np.asarray(local_moments[0], dtype=np.float64))
        for q in local_moments:
            total = total + np.asarray(q, dtype=np.float64)
        return total
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    mine = torch.from_numpy(np.ascontiguousarray(local_moments, dtype=np.float64)).to(dev)
    parts = [torch.empty_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    total = np.zeros(tuple(mine.shape))
    for p in parts:
        total = total + p.cpu().numpy()
    return total
