"""Oracle for the hyperbolic self-gravity scheme (arXiv 1602.05700) -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU reference of the wave-equation replacement of Poisson's equation (Sec. 1, Eq. HNeq.), stepped as
described in Sec. 2 and with the outer boundary conditions of Sec. 2 and Sec. 4.  The arithmetic lives in
``hg_oracle.c`` (plain C, single thread, no fused multiply-add contraction); this module only marshals numpy
arrays to it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it: the product library never does, and the two share no code.

Every function here is pinned by ``tests/test_oracle_pins.py`` against something other than itself (a DST
Poisson solve, the exact discrete plane wave, the Green's-function sum, the analytic sphere, the spherical
harmonic addition theorem, a sparse direct solve with the Robin relation, central finite differences).

The hydrodynamics that consumes -grad phi (paper Sec. 2: finite volume, HLLC, gamma = 5/3, outgoing boundaries)
lives in ``hydro_oracle.c`` and is wrapped by the ``hydro_*`` functions below; ``tests/test_hydro_pins.py`` pins
it against the exact Riemann solution, exact contact preservation, conservation, axis-permutation symmetry, the
exact momentum and energy response to a uniform field, and the polytrope's virial theorem.

Arrays: a *ghosted* array has shape (nz+2, ny+2, nx+2) with the interior at [1:-1, 1:-1, 1:-1]; an *interior*
array has shape (nz, ny, nx).  Only face ghosts are meaningful; edge and corner ghosts stay zero.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

BC_DIRICHLET = 0
BC_ROBIN = 1
BC_PERIODIC = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "hg_oracle.c"), os.path.join(_HERE, "hydro_oracle.c")]
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libhgoracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "libhgoracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle's C files with gcc (-O2, no FMA contraction, no fast-math) into oracle/_build/.  With
    openmp=True, a second library of the same files built with -fopenmp (the sweep split over the host cores), used
    only to time the oracle on all cores; the checked oracle is the single-threaded build."""
    lib = _LIB_OMP if openmp else _LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(f) for f in _SRCS):
        return lib
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           *(["-fopenmp"] if openmp else []), "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, lib)
    return lib


def run_all_cores(g: "Grid", phi: np.ndarray, phi_prev: np.ndarray, rho: np.ndarray, nsteps: int,
                  threads: int) -> None:
    """og_run from the OpenMP build (timing only): the same sub-steps as run(), split over `threads` host cores."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    lib = ctypes.CDLL(build(openmp=True))
    ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(threads))
    P = ctypes.POINTER(ctypes.c_double)
    lib.og_run.argtypes = [ctypes.POINTER(_OgGrid), P, P, P, ctypes.c_int, P]
    work = np.zeros(g.ghosted_shape)
    lib.og_run(ctypes.byref(g._s()), _p(phi), _p(phi_prev), _p(np.ascontiguousarray(rho, dtype=np.float64)),
               int(nsteps), _p(work))


class _OgGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("bc", ctypes.c_int),
                ("h", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("c", ctypes.c_double), ("G", ctypes.c_double), ("dt", ctypes.c_double)]


class _OhGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("gamma", ctypes.c_double), ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        gp = P(_OgGrid)
        lib.og_exact_sum.restype = d
        lib.og_exact_sum.argtypes = [dp, ctypes.c_size_t]
        lib.og_mean.restype = d
        lib.og_mean.argtypes = [gp, dp]
        lib.og_mass.restype = d
        lib.og_mass.argtypes = [gp, dp]
        lib.og_real_ylm.argtypes = [ctypes.c_int, d, d, d, dp]
        lib.og_moments.argtypes = [gp, dp, ctypes.c_int, dp]
        lib.og_multipole_phi.restype = d
        lib.og_multipole_phi.argtypes = [gp, ctypes.c_int, dp, d, d, d]
        lib.og_fill_multipole_ghosts.argtypes = [gp, ctypes.c_int, dp, dp]
        lib.og_fill_periodic_ghosts.argtypes = [gp, dp]
        lib.og_fill_robin_static_ghosts.argtypes = [gp, dp]
        lib.og_step.argtypes = [gp, dp, dp, dp, dp]
        lib.og_run.argtypes = [gp, dp, dp, dp, ctypes.c_int, dp]
        lib.og_accel.argtypes = [gp, dp, dp, dp, dp]
        lib.og_residual.argtypes = [gp, dp, dp, dp]
        lib.og_compare.argtypes = [gp, dp, dp, dp]
        lib.og_adjoint.argtypes = [gp, dp, ctypes.c_int, dp]
        hp = P(_OhGrid)
        lib.oh_cons_from_prim.argtypes = [hp, dp, dp]
        lib.oh_prim_from_cons.argtypes = [hp, dp, dp]
        lib.oh_hllc.argtypes = [d, dp, dp, ctypes.c_int, dp]
        lib.oh_residual.argtypes = [hp, dp, ctypes.c_void_p, dp]
        lib.oh_step.argtypes = [hp, dp, ctypes.c_void_p, d, dp]
        lib.oh_max_speed.restype = d
        lib.oh_max_speed.argtypes = [hp, dp]
        lib.oh_virial.argtypes = [hp, dp, dp, dp]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Grid:
    """Grid of nx*ny*nz cubic cells of side h; cell (i,j,k) is centred at origin + ((i,j,k) + 1/2) h."""
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple
    c: float
    G: float
    dt: float
    bc: int

    def _s(self) -> _OgGrid:
        return _OgGrid(self.nx, self.ny, self.nz, self.bc, self.h, self.origin[0], self.origin[1], self.origin[2],
                       self.c, self.G, self.dt)

    @property
    def ghosted_shape(self):
        return (self.nz + 2, self.ny + 2, self.nx + 2)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def centres(self, ghosts: bool = False):
        """Cell-centre coordinate arrays (z, y, x order of axes), interior or ghosted."""
        o = 1 if ghosts else 0
        xs = self.origin[0] + (np.arange(-o, self.nx + o) + 0.5) * self.h
        ys = self.origin[1] + (np.arange(-o, self.ny + o) + 0.5) * self.h
        zs = self.origin[2] + (np.arange(-o, self.nz + o) + 0.5) * self.h
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        return X, Y, Z


def unit_cube(n: int, c: float, G: float, cfl: float, bc: int, ny: int | None = None, nz: int | None = None) -> Grid:
    """n^3 (or n x ny x nz) cells of side 1/n, lower corner at -1/2 in every axis; dt = cfl h / (c sqrt 3)."""
    h = 1.0 / n
    return Grid(n, ny or n, nz or n, h, (-0.5, -0.5, -0.5), c, G, cfl * h / (c * np.sqrt(3.0)), bc)


def ghosted(g: Grid, interior: np.ndarray | None = None) -> np.ndarray:
    a = np.zeros(g.ghosted_shape)
    if interior is not None:
        a[1:-1, 1:-1, 1:-1] = interior
    return a


def interior(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a[1:-1, 1:-1, 1:-1])


def exact_sum(x: np.ndarray) -> float:
    """The sum of the values rounded once to the nearest double (the oracle's summation of every sum the method
    defines: moments, mass, mean)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    return _L().og_exact_sum(_p(x), x.size)


def mean(g: Grid, rho: np.ndarray) -> float:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    return _L().og_mean(ctypes.byref(g._s()), _p(rho))


def mass(g: Grid, rho: np.ndarray) -> float:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    return _L().og_mass(ctypes.byref(g._s()), _p(rho))


def real_ylm(lmax: int, x: float, y: float, z: float) -> np.ndarray:
    Y = np.zeros((lmax + 1) ** 2)
    _L().og_real_ylm(lmax, x, y, z, _p(Y))
    return Y


def moments(g: Grid, rho: np.ndarray, lmax: int) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    Q = np.zeros((lmax + 1) ** 2)
    _L().og_moments(ctypes.byref(g._s()), _p(rho), lmax, _p(Q))
    return Q


def multipole_phi(g: Grid, lmax: int, Q: np.ndarray, x: float, y: float, z: float) -> float:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    return _L().og_multipole_phi(ctypes.byref(g._s()), lmax, _p(Q), x, y, z)


def fill_multipole_ghosts(g: Grid, lmax: int, Q: np.ndarray, phi: np.ndarray) -> None:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    _L().og_fill_multipole_ghosts(ctypes.byref(g._s()), lmax, _p(Q), _p(phi))


def fill_periodic_ghosts(g: Grid, phi: np.ndarray) -> None:
    _L().og_fill_periodic_ghosts(ctypes.byref(g._s()), _p(phi))


def fill_robin_static_ghosts(g: Grid, phi: np.ndarray) -> None:
    _L().og_fill_robin_static_ghosts(ctypes.byref(g._s()), _p(phi))


def step(g: Grid, phi: np.ndarray, phi_prev: np.ndarray, rho: np.ndarray) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.zeros(g.ghosted_shape)
    _L().og_step(ctypes.byref(g._s()), _p(phi), _p(phi_prev), _p(rho), _p(out))
    return out


def run(g: Grid, phi: np.ndarray, phi_prev: np.ndarray, rho: np.ndarray, nsteps: int) -> None:
    """Advance (phi, phi_prev) in place by nsteps sub-steps."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    work = np.zeros(g.ghosted_shape)
    _L().og_run(ctypes.byref(g._s()), _p(phi), _p(phi_prev), _p(rho), int(nsteps), _p(work))


def accel(g: Grid, phi: np.ndarray):
    ax, ay, az = (np.zeros(g.shape) for _ in range(3))
    _L().og_accel(ctypes.byref(g._s()), _p(phi), _p(ax), _p(ay), _p(az))
    return ax, ay, az


def residual(g: Grid, phi: np.ndarray, rho: np.ndarray):
    """(rms, max) of Laplacian_h phi - 4 pi G (rho - rho_bar) over the interior."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.zeros(2)
    _L().og_residual(ctypes.byref(g._s()), _p(phi), _p(rho), _p(out))
    return float(out[0]), float(out[1])


def compare(g: Grid, a: np.ndarray, b: np.ndarray):
    """(rel L2, rel Linf, paper's <dphi~>) of ghosted a against ghosted b over the interior."""
    out = np.zeros(3)
    _L().og_compare(ctypes.byref(g._s()), _p(a), _p(b), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def adjoint(g: Grid, lam_T: np.ndarray, T: int) -> np.ndarray:
    """dL/drho for L depending on phi^T only, given lam_T = dL/dphi^T (interior array), after T sub-steps."""
    lam_T = np.ascontiguousarray(lam_T, dtype=np.float64)
    grad = np.zeros(g.shape)
    _L().og_adjoint(ctypes.byref(g._s()), _p(lam_T), int(T), _p(grad))
    return grad


# ---- state set-up per boundary condition (initial data as the paper's tests use it: phi = 0 or a seed) -------

def initial_state(g: Grid, rho: np.ndarray, lmax: int = 0, phi0: np.ndarray | None = None,
                  phi_prev0: np.ndarray | None = None):
    """Ghosted (phi, phi_prev) at t = 0.  Interior from the seeds (default 0); face ghosts per boundary condition:
    multipole Dirichlet data of rho, periodic copies, or the Robin static limit of the seeded interior."""
    phi = ghosted(g, phi0)
    prev = ghosted(g, phi_prev0 if phi_prev0 is not None else phi0)
    if g.bc == BC_DIRICHLET:
        Q = moments(g, rho, lmax)
        fill_multipole_ghosts(g, lmax, Q, phi)
        fill_multipole_ghosts(g, lmax, Q, prev)
    elif g.bc == BC_PERIODIC:
        fill_periodic_ghosts(g, phi)
        fill_periodic_ghosts(g, prev)
    else:
        fill_robin_static_ghosts(g, phi)
        fill_robin_static_ghosts(g, prev)
    return phi, prev


# ---- hydrodynamics consuming -grad phi (paper Sec. 2) ------------------------------------------------------------

@dataclass
class HydroGrid:
    """nx*ny*nz cells of side h for the ideal-gas hydrodynamics; fields are (5, nz, ny, nx) float64 arrays of
    conserved (rho, mx, my, mz, E) or primitive (rho, vx, vy, vz, P) variables."""
    nx: int
    ny: int
    nz: int
    h: float
    gamma: float = 5.0 / 3.0
    rho_floor: float = 0.0
    p_floor: float = 0.0

    def _s(self) -> _OhGrid:
        return _OhGrid(self.nx, self.ny, self.nz, self.h, self.gamma, self.rho_floor, self.p_floor)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def _fields(hg: HydroGrid, a, planes: int = 5) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (planes,) + hg.shape, a.shape
    return a


def hydro_cons(hg: HydroGrid, W) -> np.ndarray:
    W = _fields(hg, W)
    U = np.zeros_like(W)
    _L().oh_cons_from_prim(ctypes.byref(hg._s()), _p(W), _p(U))
    return U


def hydro_prim(hg: HydroGrid, U) -> np.ndarray:
    U = _fields(hg, U)
    W = np.zeros_like(U)
    _L().oh_prim_from_cons(ctypes.byref(hg._s()), _p(U), _p(W))
    return W


def hydro_hllc(gamma: float, wl, wr, d: int) -> np.ndarray:
    """HLLC flux along axis d (0 = x) between primitive states wl and wr (5 values each)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    F = np.zeros(5)
    _L().oh_hllc(gamma, _p(wl), _p(wr), int(d), _p(F))
    return F


def hydro_residual(hg: HydroGrid, U, A=None) -> np.ndarray:
    """L(U) = -div F / h + S(U); A = (ax, ay, az) or None."""
    U = _fields(hg, U)
    L = np.zeros_like(U)
    Ap = None if A is None else _fields(hg, A, 3)
    _L().oh_residual(ctypes.byref(hg._s()), _p(U), None if Ap is None else _p(Ap), _p(L))
    return L


def hydro_step(hg: HydroGrid, U: np.ndarray, dt: float, A=None) -> None:
    """One two-stage hydro step of dt, in place on the conserved fields U."""
    assert U.dtype == np.float64 and U.flags.c_contiguous and U.shape == (5,) + hg.shape
    Ap = None if A is None else _fields(hg, A, 3)
    work = np.zeros((10,) + hg.shape)
    _L().oh_step(ctypes.byref(hg._s()), _p(U), None if Ap is None else _p(Ap), float(dt), _p(work))


def hydro_max_speed(hg: HydroGrid, U) -> float:
    return _L().oh_max_speed(ctypes.byref(hg._s()), _p(_fields(hg, U)))


def hydro_virial(hg: HydroGrid, U, phi) -> dict:
    """The paper's virial measure over bound cells; phi is an interior (nz, ny, nx) array."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    assert phi.shape == hg.shape
    out = np.zeros(6)
    _L().oh_virial(ctypes.byref(hg._s()), _p(_fields(hg, U)), _p(phi), _p(out))
    return dict(W=out[0], U=out[1], K=out[2], VC=out[3], rho_max=out[4], M_bound=out[5])


def coupled_step(og: Grid, phi: np.ndarray, phi_prev: np.ndarray, hg: HydroGrid, U: np.ndarray, dt: float,
                 n_sub: int, lmax: int = 0) -> None:
    """One hydro step with self-gravity (Sec. 2): the wave equation advanced n_sub sub-steps with rho = U[0] held
    fixed, then the hydro step of dt with a = -grad phi of the advanced potential (both in place).  With Dirichlet
    boundaries the ghost data of both time levels are first recomputed from the step's density by the multipole
    expansion up to lmax (Sec. 4: the boundary values follow the current density)."""
    if og.bc == BC_DIRICHLET:
        Q = moments(og, U[0], lmax)
        fill_multipole_ghosts(og, lmax, Q, phi)
        fill_multipole_ghosts(og, lmax, Q, phi_prev)
    run(og, phi, phi_prev, U[0], n_sub)
    A = np.stack(accel(og, phi))
    hydro_step(hg, U, dt, A)
