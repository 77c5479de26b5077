"""torch.autograd entry points for dL/drho through the hyperbolic sub-steps (hand-written adjoint, no tape).

The time-stepper is linear in rho, so its adjoint (hg_adjoint_*) runs backward without any forward state.  Two
Functions are provided:

* ``potential(rho, grid, T)`` -- phi^T on the interior after T sub-steps from phi = 0; backward = one reverse sweep
  of T adjoint sub-steps seeded with dL/dphi^T.
* ``trajectory_loss(rho, grid, T, observe, step_loss, checkpoint_every=K)`` -- L = sum over the observed sub-steps n
  of step_loss(n, phi^n), for losses that look at many intermediate potentials.  The forward pass keeps only a
  checkpoint of the state every K sub-steps (device memory, hg_save_state); the backward pass walks the segments in
  reverse, recomputes each segment's potentials from its checkpoint, differentiates step_loss on them with torch,
  and feeds the results into the reverse sweep.  Memory: ceil(T/K) states plus the observed fields of one segment,
  against T fields for storing the whole trajectory.

Dirichlet boundary data are constants for the gradient (their dependence on rho through the multipole moments is
not differentiated).
"""
from __future__ import annotations

import math

import torch


class _Potential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, grid, T):
        grid.set_density(rho)
        grid.set_phi(torch.zeros(grid.shape, dtype=torch.float64, device=grid.device))
        grid.step(T)
        ctx.grid, ctx.T, ctx.rho_dtype = grid, int(T), rho.dtype
        return grid.phi(torch.float64)

    @staticmethod
    def backward(ctx, g_phi):
        grid = ctx.grid
        grid.adjoint_reset()
        grid.adjoint_inject(g_phi.contiguous().to(torch.float64))
        grid.adjoint_step(ctx.T)
        return grid.adjoint_grad(torch.float64).to(ctx.rho_dtype), None, None


def potential(rho: torch.Tensor, grid, T: int) -> torch.Tensor:
    """phi^T (float64, interior) after T sub-steps from phi = 0 with density rho; differentiable in rho."""
    return _Potential.apply(rho, grid, T)


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, grid, T, observe, step_loss, K):
        T = int(T)
        K = max(1, int(K))
        observe = sorted(set(int(n) for n in observe if 1 <= int(n) <= T))
        grid.set_density(rho)
        grid.set_phi(torch.zeros(grid.shape, dtype=torch.float64, device=grid.device))
        nbytes = grid.state_bytes()
        ckpts = []
        total = torch.zeros((), dtype=torch.float64, device=grid.device)
        obs = set(observe)
        n = 0
        while n < T:
            buf = torch.empty(nbytes, dtype=torch.uint8, device=grid.device)
            ckpts.append((n, grid.save_state(buf)))
            end = min(n + K, T)
            while n < end:
                nxt = min([m for m in observe if m > n and m <= end] or [end])
                grid.step(nxt - n)
                n = nxt
                if n in obs:
                    with torch.no_grad():
                        total = total + step_loss(n, grid.phi(torch.float64))
        ctx.grid, ctx.T, ctx.K, ctx.observe, ctx.step_loss = grid, T, K, observe, step_loss
        ctx.ckpts, ctx.rho_dtype = ckpts, rho.dtype
        ctx.memory = {"checkpoints": len(ckpts), "checkpoint_bytes": len(ckpts) * nbytes,
                      "full_trajectory_bytes": T * grid.nx * grid.ny * grid.nz * 8}
        return total

    @staticmethod
    def backward(ctx, gL):
        grid, obs = ctx.grid, set(ctx.observe)
        grid.adjoint_reset()
        for start, buf in reversed(ctx.ckpts):
            end = min(start + ctx.K, ctx.T)
            seg = [m for m in ctx.observe if start < m <= end]
            fields = {}
            if seg:  # recompute the observed potentials of this segment from its checkpoint
                grid.load_state(buf)
                n = start
                for m in seg:
                    grid.step(m - n)
                    n = m
                    fields[m] = grid.phi(torch.float64)
            m = end
            while m > start:
                if m in obs:
                    phi = fields.pop(m).requires_grad_(True)
                    with torch.enable_grad():
                        (g,) = torch.autograd.grad(ctx.step_loss(m, phi), phi)
                    grid.adjoint_inject((g * gL).contiguous())
                # reverse sub-steps down to the next observed level (or the segment start)
                nxt = max([o for o in seg if o < m] or [start])
                grid.adjoint_step(m - nxt)
                m = nxt
        return grid.adjoint_grad(torch.float64).to(ctx.rho_dtype), None, None, None, None, None


def trajectory_loss(rho, grid, T, observe, step_loss, checkpoint_every=None):
    """sum over n in `observe` of step_loss(n, phi^n) after sub-steps from phi = 0; differentiable in rho.

    checkpoint_every=K keeps a state checkpoint every K sub-steps and recomputes segments in the backward pass
    (default: K = ceil(sqrt(T)))."""
    K = checkpoint_every or max(1, int(math.ceil(math.sqrt(T))))
    return _Trajectory.apply(rho, grid, T, tuple(observe), step_loss, K)


def trilinear_probe_weights(grid, points: torch.Tensor):
    """(indices, weights) for trilinear interpolation of a cell-centred field at points (P, 3): phi(x_p) =
    sum_k weights[p, k] * phi.view(-1)[indices[p, k]].  Used by probe losses; plain torch."""
    dev = grid.device
    pts = points.to(device=dev, dtype=torch.float64)
    o = torch.tensor(grid.origin, dtype=torch.float64, device=dev)
    u = (pts - o) / grid.h - 0.5  # cell-index coordinates
    i0 = torch.floor(u).to(torch.long)
    f = u - i0
    n = torch.tensor([grid.nx, grid.ny, grid.nz], device=dev)
    idx, wts = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                d = torch.tensor([dx, dy, dz], device=dev)
                c = torch.minimum(torch.maximum(i0 + d, torch.zeros_like(i0)), n - 1)
                w = torch.prod(torch.where(d.bool(), f, 1.0 - f), dim=1)
                idx.append((c[:, 2] * grid.ny + c[:, 1]) * grid.nx + c[:, 0])
                wts.append(w)
    return torch.stack(idx, 1), torch.stack(wts, 1)
