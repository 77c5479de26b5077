"""Adjoint of the sub-stepping on the GPU: against the oracle's discrete adjoint, central finite differences (exact
for a loss quadratic in rho), the dot-product identity, and checkpointed against unsegmented reverse sweeps."""
import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from paper_1602_05700_gb300 import autograd as HA  # noqa: E402
from tests.test_gpu_parity import BC_PAIRS, check, pair, robin_cfl  # noqa: E402


@pytest.mark.parametrize("prec", ["f64", "f32k"])
@pytest.mark.parametrize("bc", ["multipole", "robin", "periodic", "dirichlet"])
def test_adjoint_matches_oracle(prec, bc):
    nx, ny, nz = 35, 29, 23
    h = 1.0 / 32
    g, og = pair(nx, ny, nz, h, bc, prec, lmax=2 if bc == "multipole" else 0,
                 cfl=robin_cfl(nx, ny, nz, h) if bc == "robin" else 0.7)
    T = 30
    lam = I.noise(og.shape, 301, -1.0, 1.0)
    g.adjoint_reset()
    g.adjoint_inject(torch.from_numpy(lam).cuda())
    g.adjoint_step(T)
    got = g.adjoint_grad().cpu().numpy()
    want = O.adjoint(og, lam, T)
    check(prec, got, want, f"adjoint {bc}")
    # a second reset starts from scratch
    g.adjoint_reset()
    g.adjoint_inject(lam)  # from host memory this time
    g.adjoint_step(T)
    assert np.array_equal(g.adjoint_grad().cpu().numpy(), got)
    # the one-call terminal-loss form gives the same result, from device and from host buffers
    assert np.array_equal(g.adjoint(torch.from_numpy(lam).cuda(), T).cpu().numpy(), got)
    assert np.array_equal(g.adjoint(lam, T).numpy(), got)


def _probe_loss(grid, T, probes, target):
    idx, w = HA.trilinear_probe_weights(grid, probes)

    def loss(rho):
        phi = HA.potential(rho, grid, T)
        vals = (phi.reshape(-1)[idx] * w).sum(1)
        return ((vals - target) ** 2).sum()

    return loss, idx, w


def test_potential_gradient_against_finite_differences_f64():
    """Config-5 shape at reduced size: FP64, 4 blobs (seed 3), 64 probes in |x| < 0.4, target from the seed-4
    density, loss sum (phi^T(x_p) - target_p)^2.  L is quadratic in rho, so central differences are exact up to
    rounding for any step."""
    n, T = 48, 120
    grid = hg.Grid.unit_cube(n, precision="f64", bc="robin")
    rho = torch.from_numpy(I.blob_density(n, I.draw_blobs(4, 3))).cuda()
    rho_t = torch.from_numpy(I.blob_density(n, I.draw_blobs(4, 4))).cuda()
    probes = torch.from_numpy(I.probes(64, 11))
    idx, w = HA.trilinear_probe_weights(grid, probes)
    with torch.no_grad():
        target = (HA.potential(rho_t, grid, T).reshape(-1)[idx] * w).sum(1)
    loss, _, _ = _probe_loss(grid, T, probes, target)
    r = rho.clone().requires_grad_(True)
    L = loss(r)
    L.backward()
    grad = r.grad.detach().cpu().numpy()
    rng = np.random.default_rng(5)
    cells = [tuple(rng.integers(0, n, 3)) for _ in range(6)]
    # include cells next to probes, where the gradient is large
    for p in idx[:4, 0].cpu().numpy():
        cells.append((p // (n * n), (p // n) % n, p % n))
    eps = 1e-2
    for k, j, i in cells:
        with torch.no_grad():
            rp = rho.clone()
            rp[k, j, i] += eps
            rm = rho.clone()
            rm[k, j, i] -= eps
            fd = (loss(rp) - loss(rm)).item() / (2 * eps)
        assert abs(fd - grad[k, j, i]) <= 1e-6 * np.abs(grad).max(), (k, j, i, fd, grad[k, j, i])


@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_dot_product_identity(prec):
    n, T = 40, 60
    grid = hg.Grid.unit_cube(n, precision=prec, bc="robin")
    drho = torch.from_numpy(I.noise((n, n, n), 51, -1.0, 1.0)).cuda()
    mu = torch.from_numpy(I.noise((n, n, n), 52, -1.0, 1.0)).cuda()
    phi = HA.potential(drho, grid, T)  # linear part: zero initial state, Robin boundary has no data
    lhs = float((phi * mu).sum())
    grid.adjoint_reset()
    grid.adjoint_inject(mu)
    grid.adjoint_step(T)
    rhs = float((drho * grid.adjoint_grad()).sum())
    tol = 1e-11 if prec == "f64" else 1e-5
    assert abs(lhs - rhs) <= tol * abs(lhs)


@pytest.mark.parametrize("K", [7, 50])
def test_checkpointed_trajectory_loss(K):
    """Loss on every 10th potential; the checkpointed reverse sweep (segments of K) gives the gradient of the
    unsegmented one and of central differences."""
    n, T = 32, 60
    grid = hg.Grid.unit_cube(n, precision="f64", bc="robin")
    rho = torch.from_numpy(I.blob_density(n, I.draw_blobs(3, 8))).cuda()
    probes = torch.from_numpy(I.probes(16, 12))
    idx, w = HA.trilinear_probe_weights(grid, probes)
    obs = list(range(10, T + 1, 10))

    def step_loss(m, phi):
        vals = (phi.reshape(-1)[idx] * w).sum(1)
        return (m / T) * (vals ** 2).sum()

    grads = []
    for k in (K, T):
        r = rho.clone().requires_grad_(True)
        L = HA.trajectory_loss(r, grid, T, obs, step_loss, checkpoint_every=k)
        L.backward()
        grads.append(r.grad.detach().cpu().numpy())
    assert np.allclose(grads[0], grads[1], rtol=0, atol=1e-13 * np.abs(grads[1]).max())
    cell = tuple(int(v) for v in np.unravel_index(np.argmax(np.abs(grads[0])), grads[0].shape))
    eps = 1e-2
    with torch.no_grad():
        rp = rho.clone()
        rp[cell] += eps
        rm = rho.clone()
        rm[cell] -= eps
        fd = (HA.trajectory_loss(rp, grid, T, obs, step_loss, K) - HA.trajectory_loss(rm, grid, T, obs, step_loss,
                                                                                      K)).item() / (2 * eps)
    assert abs(fd - grads[0][cell]) <= 1e-6 * abs(grads[0][cell])
