"""hg_moments_noalloc: the multipole moments for callers that may not allocate GPU memory.

Such a caller passes its own density and output buffers and gets the same FP64 moments that a grid computes in
hg_set_density, with the scratch taken from a fixed array inside the library.  Checked through the C ABI against
hg_get_moments (the existing entry point) and against the CPU oracle's moments, at the FP64 tolerance of the
other tests, on consecutive calls (the shared scratch must not carry anything over from one call to the next) and
with the result in device or host memory.  This file is collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1602_05700_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1602_05700_gb300 as hg  # noqa: E402
from paper_1602_05700_gb300 import _lib  # noqa: E402

TOL = 1e-12  # relative, as for every FP64 result in the GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    hg.build()


def reference(n, rho, lmax):
    g = hg.Grid.unit_cube(n, precision="f64", bc="multipole", lmax=lmax)
    g.set_density(rho)
    Q = g.moments()
    g.free()
    return Q


def noalloc(rho, lmax, n, on_device):
    L = _lib.lib()
    origin = (ctypes.c_double * 3)(-0.5, -0.5, -0.5)
    nq = (lmax + 1) ** 2
    code = _lib.HG_DT_F64 if rho.dtype == torch.float64 else _lib.HG_DT_F32
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if on_device:
        out = torch.full((nq,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.hg_moments_noalloc(ctypes.c_void_p(rho.data_ptr()), code, n, n, n, 1.0 / n, origin, lmax,
                                  ctypes.c_void_p(out.data_ptr()), 1, stream)
        _lib.check(rc)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    out = np.full(nq, np.nan)
    rc = L.hg_moments_noalloc(ctypes.c_void_p(rho.data_ptr()), code, n, n, n, 1.0 / n, origin, lmax,
                              ctypes.c_void_p(out.ctypes.data), 0, stream)
    _lib.check(rc)
    return out


def close(a, b):
    return np.abs(a - b).max() <= TOL * np.abs(b).max()


def oracle_moments(n, rho, lmax):
    return O.moments(O.unit_cube(n, 1.0, 1.0, 0.5, O.BC_DIRICHLET), rho.double().cpu().numpy(), lmax)


def test_matches_grid_moments_on_consecutive_calls():
    n = 48
    rho = torch.from_numpy(I.sphere_density(n) + I.blob_density(n, I.draw_blobs(8, 1))).cuda()
    Q4 = reference(n, rho, 4)
    assert close(Q4, oracle_moments(n, rho, 4))
    first = noalloc(rho, 4, n, on_device=True)
    second = noalloc(rho, 4, n, on_device=True)
    O4 = oracle_moments(n, rho, 4)
    assert close(first, Q4) and close(second, Q4)
    assert close(first, O4) and close(second, O4)
    assert close(noalloc(rho, 4, n, on_device=False), O4)
    # a different density and order right after: nothing of the previous calls may leak into the result
    rho2 = torch.from_numpy(I.blob_density(n, I.draw_blobs(3, 9))).to(torch.float32).cuda()
    Q8 = reference(n, rho2, 8)
    O8 = oracle_moments(n, rho2, 8)
    assert close(Q8, O8)
    for on_device in (True, False):
        got = noalloc(rho2, 8, n, on_device=on_device)
        assert close(got, Q8) and close(got, O8)
    assert close(noalloc(rho, 4, n, on_device=True), Q4)


def test_rejects_order_beyond_the_scratch():
    n = 8
    rho = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
    L = _lib.lib()
    origin = (ctypes.c_double * 3)(-0.5, -0.5, -0.5)
    out = np.zeros(100)
    rc = L.hg_moments_noalloc(ctypes.c_void_p(rho.data_ptr()), _lib.HG_DT_F64, n, n, n, 1.0 / n, origin,
                              _lib.HG_MAX_LMAX + 1, ctypes.c_void_p(out.ctypes.data), 0, None)
    assert rc == _lib.HG_ERR_ARG
    assert b"lmax" in L.hg_last_error()
    assert L.hg_moments_noalloc(None, _lib.HG_DT_F64, n, n, n, 1.0 / n, origin, 2, ctypes.c_void_p(out.ctypes.data), 0,
                                None) == _lib.HG_ERR_ARG
