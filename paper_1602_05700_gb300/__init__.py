"""Python binding of the GB300 hyperbolic self-gravity library (arXiv 1602.05700).

A thin layer over the C ABI of include/hg.h: it turns tensors and arrays into pointers, sizes and flags.  Every
step of the method runs in the CUDA kernels of ``csrc/``; PyTorch only provides device memory and streams.

    import torch, paper_1602_05700_gb300 as hg
    g = hg.Grid.unit_cube(256, c=1.0, G=1.0, cfl=0.5, precision="f32k", bc="robin")
    g.set_density(rho)           # (nz, ny, nx) tensor or array, rho frozen over the sub-steps (Sec. 2)
    g.step(20)                   # k_g wave sub-steps per hydro step (Sec. 2)
    ax, ay, az = g.accel()       # -grad phi for the hydro step

The hydrodynamics that consumes it (Sec. 2: finite volume, HLLC, gamma = 5/3, outgoing boundaries) is ``Hydro``:

    H = hg.Hydro(g.nx, g.ny, g.nz, g.h, dtype="f32")
    H.set_primitive(W)           # (5, nz, ny, nx): rho, vx, vy, vz, P
    H.step(dt, g, n_sub)         # rho -> g, n_sub wave sub-steps, -grad phi, two Runge-Kutta stages
    H.virial(g)                  # the paper's VC over bound cells
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (HG_BC_DIRICHLET_ANALYTIC, HG_BC_DIRICHLET_MULTIPOLE, HG_BC_PERIODIC, HG_BC_ROBIN, HG_DT_F32,
                   HG_DT_F64, HG_MAX_LMAX, HG_MAX_TEMPORAL_DEPTH, HG_PREC_F32K, HG_PREC_F64, HGError)

BC = {"dirichlet": HG_BC_DIRICHLET_ANALYTIC, "dirichlet_analytic": HG_BC_DIRICHLET_ANALYTIC,
      "multipole": HG_BC_DIRICHLET_MULTIPOLE, "dirichlet_multipole": HG_BC_DIRICHLET_MULTIPOLE,
      "robin": HG_BC_ROBIN, "periodic": HG_BC_PERIODIC}
PREC = {"f32k": HG_PREC_F32K, "f64": HG_PREC_F64}

__all__ = ["Grid", "Batch", "Hydro", "HGError", "BC", "PREC", "build", "is_debug_build"]


def build(force: bool = False, debug: bool = False) -> str:
    """Build the CUDA library in-tree (debug=True: the HG_DEBUG variant with index checks)."""
    from .builder import build as _b
    return _b(force=force, debug=debug)


def is_debug_build() -> bool:
    """Whether the loaded library is the HG_DEBUG variant (HG_DEBUG=1 in the environment at import)."""
    return bool(_lib.lib().hg_is_debug_build())


def probe_rate(kind: str) -> dict:
    """Measured arithmetic rate of the current GPU (hg_probe_rate): kind "f64", "f32" or "f32x2" (the packed pair).
    Returns thread instructions/s and multiply-adds/s."""
    code = {"f64": 0, "f32": 1, "f32x2": 2}[kind]
    ins, ops = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.lib().hg_probe_rate(code, ctypes.byref(ins), ctypes.byref(ops)))
    return {"instr_per_s": ins.value, "fma_per_s": ops.value}


def _torch():
    import torch
    return torch


def _buffer(x, want_dtype=None):
    """(pointer, dtype code, on_device, keepalive) for a torch tensor or numpy array holding nz*ny*nx values."""
    try:
        torch = _torch()
        is_tensor = isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_tensor = False
    if is_tensor:
        t = x
        if t.dtype not in (torch.float32, torch.float64):
            t = t.to(torch.float64)
        t = t.contiguous()
        code = HG_DT_F64 if t.dtype == torch.float64 else HG_DT_F32
        return ctypes.c_void_p(t.data_ptr()), code, 1 if t.is_cuda else 0, t
    a = np.asarray(x)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    code = HG_DT_F64 if a.dtype == np.float64 else HG_DT_F32
    return ctypes.c_void_p(a.ctypes.data), code, 0, a


def _writable_host(x) -> bool:
    """True for a contiguous float32/float64 host tensor or array (one the library can write in place)."""
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return not x.is_cuda and x.is_contiguous() and x.dtype in (torch.float32, torch.float64)
    return isinstance(x, np.ndarray) and x.flags.c_contiguous and x.flags.writeable and \
        x.dtype in (np.float32, np.float64)


class Grid:
    """One grid of nx*ny*nz cells of side h (lower corner `origin`), wave speed c, constant G, sub-step dt."""

    def __init__(self, nx, ny, nz, h, origin, c, G, dt, precision="f32k", bc="robin", lmax=0, stream=None,
                 z_interfaces=0):
        """z_interfaces (bits 0 / 1): the -z / +z face is an interface to a neighbouring slab (hg_init_slab)."""
        torch = _torch()
        L = _lib.lib()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        handle = ctypes.c_void_p()
        org = (ctypes.c_double * 3)(*[float(o) for o in origin])
        prec = PREC[precision] if isinstance(precision, str) else int(precision)
        bcc = BC[bc] if isinstance(bc, str) else int(bc)
        if z_interfaces:
            _lib.check(L.hg_init_slab(ctypes.byref(handle), int(nx), int(ny), int(nz), float(h), org, float(c),
                                      float(G), float(dt), prec, bcc, int(lmax), ctypes.c_void_p(stream.cuda_stream),
                                      int(z_interfaces)))
        else:
            _lib.check(L.hg_init_grid(ctypes.byref(handle), int(nx), int(ny), int(nz), float(h), org, float(c),
                                      float(G), float(dt), prec, bcc, int(lmax), ctypes.c_void_p(stream.cuda_stream)))
        self._h = handle
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.origin = tuple(float(o) for o in origin)
        self.c, self.G, self.dt = float(c), float(G), float(dt)
        self.precision, self.bc, self.lmax = prec, bcc, int(lmax)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._io_keep = []  # buffers of io_step calls not yet covered by io_wait

    @classmethod
    def unit_cube(cls, n, c=1.0, G=1.0, cfl=0.5, precision="f32k", bc="robin", lmax=0, ny=None, nz=None, stream=None):
        """n cells per side of [-1/2, 1/2] (h = 1/n), dt = cfl h / (c sqrt 3)."""
        h = 1.0 / n
        return cls(n, ny or n, nz or n, h, (-0.5, -0.5, -0.5), c, G, cfl * h / (c * np.sqrt(3.0)), precision, bc,
                   lmax, stream)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def handle(self):
        if self._h is None:
            raise HGError(-1, "grid was freed")
        return self._h

    def set_density(self, rho):
        p, code, dev, keep = _buffer(rho)
        self._check_size(keep)
        _lib.check(_lib.lib().hg_set_density(self.handle, p, code, dev))

    def set_phi(self, phi, phi_prev=None):
        p, code, dev, keep = _buffer(phi)
        self._check_size(keep)
        if phi_prev is not None:
            q, code2, dev2, keep2 = _buffer(phi_prev, code)
            self._check_size(keep2)
            if code2 != code or dev2 != dev:
                raise HGError(-1, "phi and phi_prev must have the same dtype and device")
        else:
            q, keep2 = ctypes.c_void_p(0), None
        _lib.check(_lib.lib().hg_set_phi(self.handle, p, q, code, dev))

    def step(self, n=1):
        _lib.check(_lib.lib().hg_step(self.handle, int(n)))

    def set_temporal_depth(self, k):
        _lib.check(_lib.lib().hg_set_temporal_depth(self.handle, int(k)))

    def set_temporal_exact(self, exact=True):
        """Fused sub-steps bit-identical to single sweeps (their inner levels round the compensation as a store
        would); off by default, where the inner levels keep it as a float."""
        _lib.check(_lib.lib().hg_set_temporal_exact(self.handle, 1 if exact else 0))

    def set_block_depth(self, planes):
        """z planes per block of the single-sweep kernel (0 = built-in rule); results do not depend on it."""
        _lib.check(_lib.lib().hg_set_block_depth(self.handle, int(planes)))

    def accel(self, dtype=None, out=None):
        """-grad phi^n as three (nz, ny, nx) device tensors (written into `out` when given)."""
        torch = _torch()
        if out is None:
            dtype = dtype or (torch.float64 if self.precision == HG_PREC_F64 else torch.float32)
            out = [torch.empty(self.shape, dtype=dtype, device=self.device) for _ in range(3)]
        else:
            dtype = out[0].dtype
            for t in out:
                if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype and tuple(t.shape) == self.shape):
                    raise HGError(-1, "accel outputs must be contiguous device tensors of the grid shape, one dtype")
        code = HG_DT_F64 if dtype == torch.float64 else HG_DT_F32
        _lib.check(_lib.lib().hg_accel(self.handle, *[ctypes.c_void_p(t.data_ptr()) for t in out], code))
        return tuple(out)

    def io_step(self, rho=None, n=1, out=None):
        """One hydro step with host buffers, pipelined: upload rho (host, nz*ny*nx), n sub-steps, -grad phi into
        `out` (three host arrays or tensors of the grid shape, one dtype).  Returns before the GPU is done; the
        buffers are in use until io_wait covers this call (io_wait(1) after each call keeps one step in flight)."""
        keep = []
        rp, rcode = ctypes.c_void_p(0), HG_DT_F32
        if rho is not None:
            rp, rcode, dev, k = _buffer(rho)
            self._check_size(k)
            if dev:
                raise HGError(-1, "io_step takes host buffers (use set_density for device data)")
            keep.append(k)
        ptrs, acode = [ctypes.c_void_p(0)] * 3, HG_DT_F32
        if out is not None:
            ptrs, codes = [], set()
            for o in out:
                if not _writable_host(o):
                    raise HGError(-1, "io_step outputs must be contiguous float32/float64 host buffers")
                p, code, _, k = _buffer(o)
                self._check_size(k)
                ptrs.append(p)
                codes.add(code)
                keep.append(k)
            if len(ptrs) != 3 or len(codes) != 1:
                raise HGError(-1, "io_step takes three outputs of one dtype")
            acode = codes.pop()
        _lib.check(_lib.lib().hg_io_step(self.handle, rp, rcode, int(n), *ptrs, acode))
        self._io_keep.append(keep)

    def check_bounded_wait(self):
        """Run the kernels' bounded-wait diagnostic (a wait that cannot complete must give up and be reported)."""
        _lib.check(_lib.lib().hg_check_bounded_wait(self.handle))

    def check_bounds(self):
        """Debug builds: run the index-check diagnostic (an index past the array must be caught and reported as
        HG_ERR_BOUNDS, with nothing stored).  A release build raises HGError(HG_ERR_STATE)."""
        _lib.check(_lib.lib().hg_check_bounds(self.handle))

    def io_wait(self, keep=0):
        """Block until all but the newest `keep` io_step calls are done (their outputs are then filled)."""
        _lib.check(_lib.lib().hg_io_wait(self.handle, int(keep)))
        while len(self._io_keep) > keep:
            self._io_keep.pop(0)

    def phi(self, dtype=None, device="cuda"):
        """phi^n on the interior as an (nz, ny, nx) tensor (device) or numpy array (device='cpu')."""
        torch = _torch()
        dtype = dtype or torch.float64
        code = HG_DT_F64 if dtype == torch.float64 else HG_DT_F32
        if device == "cpu":
            out = np.empty(self.shape, dtype=np.float64 if code == HG_DT_F64 else np.float32)
            _lib.check(_lib.lib().hg_get_phi(self.handle, ctypes.c_void_p(out.ctypes.data), code, 0))
            return out
        out = torch.empty(self.shape, dtype=dtype, device=self.device)
        _lib.check(_lib.lib().hg_get_phi(self.handle, ctypes.c_void_p(out.data_ptr()), code, 1))
        return out

    def phi_ghosted(self) -> np.ndarray:
        out = np.empty((self.nz + 2, self.ny + 2, self.nx + 2))
        _lib.check(_lib.lib().hg_get_phi_ghosted(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def stats(self, check=True) -> dict:
        s = _lib.hg_stats()
        rc = _lib.lib().hg_get_stats(self.handle, ctypes.byref(s))
        if check:
            _lib.check(rc)
        return {k: getattr(s, k) for k, _ in _lib.hg_stats._fields_} | {"rc": rc}

    def set_boundary_moments(self, Q) -> None:
        """Dirichlet modes: face ghosts from given moments (e.g. the sum of several slabs' own moments)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        _lib.check(_lib.lib().hg_set_boundary_moments(self.handle, Q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def moments(self) -> np.ndarray:
        nq = (self.lmax + 1) ** 2 if self.bc == HG_BC_DIRICHLET_MULTIPOLE else 1
        out = np.zeros(nq)
        _lib.check(_lib.lib().hg_get_moments(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def compare(self, phi_P):
        """(rel L2, rel Linf, the paper's <dphi~>) of phi^n against a reference potential (Sec. 4)."""
        torch = _torch()
        if isinstance(phi_P, torch.Tensor):
            t = phi_P.to(torch.float64).contiguous()
            p, dev, keep = ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, t
        else:
            keep = np.ascontiguousarray(phi_P, dtype=np.float64)
            p, dev = ctypes.c_void_p(keep.ctypes.data), 0
        self._check_size(keep)
        out = (ctypes.c_double * 3)()
        _lib.check(_lib.lib().hg_compare(self.handle, p, dev, out))
        return float(out[0]), float(out[1]), float(out[2])

    def state_bytes(self) -> int:
        return int(_lib.lib().hg_state_bytes(self.handle))

    def save_state(self, out=None):
        """Checkpoint: bytes in host memory, or into `out` (a uint8 device tensor of state_bytes())."""
        if out is not None:
            _lib.check(_lib.lib().hg_save_state(self.handle, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        buf = ctypes.create_string_buffer(self.state_bytes())
        _lib.check(_lib.lib().hg_save_state(self.handle, buf, 0))
        return buf.raw

    def load_state(self, blob) -> None:
        torch = _torch()
        if isinstance(blob, torch.Tensor):
            _lib.check(_lib.lib().hg_load_state(self.handle, ctypes.c_void_p(blob.data_ptr()), 1))
            return
        buf = ctypes.create_string_buffer(blob, len(blob))
        _lib.check(_lib.lib().hg_load_state(self.handle, buf, 0))

    # ---- adjoint (see hg.h) ----
    def adjoint_reset(self):
        _lib.check(_lib.lib().hg_adjoint_reset(self.handle))

    def adjoint_inject(self, dL_dphi):
        p, code, dev, keep = _buffer(dL_dphi)
        self._check_size(keep)
        _lib.check(_lib.lib().hg_adjoint_inject(self.handle, p, code, dev))

    def adjoint_step(self, n=1):
        _lib.check(_lib.lib().hg_adjoint_step(self.handle, int(n)))

    def adjoint_grad(self, dtype=None):
        """dL/drho as an (nz, ny, nx) device tensor."""
        torch = _torch()
        dtype = dtype or torch.float64
        out = torch.empty(self.shape, dtype=dtype, device=self.device)
        code = HG_DT_F64 if dtype == torch.float64 else HG_DT_F32
        _lib.check(_lib.lib().hg_adjoint_grad(self.handle, ctypes.c_void_p(out.data_ptr()), code, 1))
        return out

    def adjoint(self, dL_dphiT, T):
        """dL/drho for L = L(phi^T) after T sub-steps, given dL/dphi^T, in one call (hg_adjoint)."""
        torch = _torch()
        p, code, dev, keep = _buffer(dL_dphiT)
        self._check_size(keep)
        out = torch.empty(self.shape, dtype=torch.float64 if code == HG_DT_F64 else torch.float32,
                          device=self.device if dev else "cpu")
        _lib.check(_lib.lib().hg_adjoint(self.handle, p, int(T), ctypes.c_void_p(out.data_ptr()), code, dev))
        return out

    def profile(self, enable=True):
        _lib.check(_lib.lib().hg_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """(sub-step kernel ms, timed launches, total kernel launches) since the last read."""
        ms, n, tot = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        _lib.check(_lib.lib().hg_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(tot)))
        return ms.value, n.value, tot.value

    def sync(self):
        _lib.check(_lib.lib().hg_sync(self.handle))

    def free(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().hg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _check_size(self, a):
        n = a.numel() if hasattr(a, "numel") else a.size
        if n != self.nx * self.ny * self.nz:
            raise HGError(-1, f"array has {n} values, grid has {self.nx * self.ny * self.nz} cells")


class Batch:
    """Several grids advanced together: one batched launch per sub-step, replayed from a CUDA graph."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g.handle for g in self.grids])
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().hg_batch_create(arr, len(self.grids), ctypes.byref(h)))
        self._h = h

    def step(self, n=1):
        _lib.check(_lib.lib().hg_batch_step(self._h, int(n)))

    def set_split(self, mode):
        """Pin the launch mode: True = one launch per precision class per sub-step, False = one launch for both,
        None = autotuned (the default).  Results do not depend on it."""
        m = -1 if mode is None else (1 if mode else 0)
        _lib.check(_lib.lib().hg_batch_set_split(self._h, m))

    def info(self):
        zb, nb = ctypes.c_int(), ctypes.c_longlong()
        _lib.check(_lib.lib().hg_batch_info(self._h, ctypes.byref(zb), ctypes.byref(nb)))
        t = (ctypes.c_int * 4)()
        _lib.check(_lib.lib().hg_batch_tuning(self._h, t))
        return {"z_planes_per_block": zb.value, "blocks_per_substep": nb.value,
                "f64_tile_rows": "per grid (128 or 32 cells)" if t[1] == 0 else "128 cells",
                "f32_z_planes_per_block": t[2], "precisions_in_separate_launches": bool(t[3])}

    def free(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().hg_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


HYDRO_DT = {"f32": HG_DT_F32, "f64": HG_DT_F64}


class Hydro:
    """Ideal-gas hydro state on nx*ny*nz cells of side h (include/hg_hydro.h): conserved (rho, mx, my, mz, E) in
    5 planes, stepped with the gravity of a matching Grid on the same stream."""

    def __init__(self, nx, ny, nz, h, gamma=5.0 / 3.0, rho_floor=0.0, p_floor=0.0, dtype="f32", stream=None):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.dtype = HYDRO_DT[dtype] if isinstance(dtype, str) else int(dtype)
        handle = ctypes.c_void_p()
        _lib.check(_lib.lib().hg_hydro_init(ctypes.byref(handle), int(nx), int(ny), int(nz), float(h), float(gamma),
                                            float(rho_floor), float(p_floor), self.dtype,
                                            ctypes.c_void_p(stream.cuda_stream)))
        self._h = handle
        self.nx, self.ny, self.nz, self.h, self.gamma = int(nx), int(ny), int(nz), float(h), float(gamma)
        self.device = torch.device("cuda", torch.cuda.current_device())

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)

    @property
    def handle(self):
        if self._h is None:
            raise HGError(-1, "hydro state was freed")
        return self._h

    def _fields(self, x):
        p, code, dev, keep = _buffer(x)
        n = keep.numel() if hasattr(keep, "numel") else keep.size
        if n != 5 * self.nx * self.ny * self.nz:
            raise HGError(-1, f"field set has {n} values, expected 5 x {self.nx * self.ny * self.nz}")
        return p, code, dev, keep

    def set_primitive(self, W):
        p, code, dev, keep = self._fields(W)
        _lib.check(_lib.lib().hg_hydro_set_primitive(self.handle, p, code, dev))

    def set_state(self, U):
        p, code, dev, keep = self._fields(U)
        _lib.check(_lib.lib().hg_hydro_set_state(self.handle, p, code, dev))

    def state(self, device="cuda"):
        torch = _torch()
        t = torch.empty(self.shape, dtype=torch.float64 if self.dtype == HG_DT_F64 else torch.float32,
                        device=self.device if device == "cuda" else "cpu")
        _lib.check(_lib.lib().hg_hydro_get_state(self.handle, ctypes.c_void_p(t.data_ptr()), self.dtype,
                                                 1 if t.is_cuda else 0))
        return t

    def max_speed(self) -> float:
        s = ctypes.c_double()
        _lib.check(_lib.lib().hg_hydro_max_speed(self.handle, ctypes.byref(s)))
        return s.value

    def step(self, dt, grid=None, n_sub=0):
        _lib.check(_lib.lib().hg_hydro_step(self.handle, grid.handle if grid is not None else None, float(dt),
                                            int(n_sub)))

    def virial(self, grid) -> dict:
        out = (ctypes.c_double * 6)()
        _lib.check(_lib.lib().hg_hydro_virial(self.handle, grid.handle, out))
        return dict(W=out[0], U=out[1], K=out[2], VC=out[3], rho_max=out[4], M_bound=out[5])

    def launches(self) -> int:
        n = ctypes.c_longlong()
        _lib.check(_lib.lib().hg_hydro_launches(self.handle, ctypes.byref(n)))
        return n.value

    def profile(self, enable=True):
        _lib.check(_lib.lib().hg_hydro_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        """(summed stage-kernel ms, stage launches) since the last read; resets both."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _lib.check(_lib.lib().hg_hydro_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def free(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().hg_hydro_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
