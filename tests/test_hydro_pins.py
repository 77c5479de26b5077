"""Pins of the hydrodynamics oracle (paper Sec. 2: finite volume, HLLC, ideal gas, outgoing boundaries, gravity
as the source -rho grad phi) and of the polytrope input, against what mathematics and textbooks fix:

* exact Riemann solution of Sod's shock tube (written here from the textbook wave curves), first-order L1
  convergence, along every axis                                      -> flux, reconstruction, update, index order
* the same 1-D problem along x, y and z gives bit-identical fields   -> transposed strides, per-axis velocity
* HLLC: consistency F(w, w) = physical flux, upwinding for supersonic states, an isolated stationary contact kept
  to rounding (an HLL flux would smear it)                            -> the star states and the contact speed
* smooth advection converges at second order (error ratio > 3.5 per halving) -> limiter, two-stage integrator
* conservation of mass, momentum and energy to rounding                -> flux differencing, boundary
* a strong blast stays positive and conservative                       -> robustness of the limiter and solver
* uniform field on a uniform gas: exact Heun response m = rho a dt, E - E0 = rho |a|^2 dt^2 / 2 -> source terms
* characteristic speed of a hand-computed state                       -> the c_g normalisation
* Lane-Emden closed forms (n = 0, 1, 5) and textbook constants (n = 1.5, 3) -> the polytrope input
* the polytrope's atmosphere in hydrostatic balance on its own, of negligible mass -> the atmosphere input
* the polytrope's discrete Laplacian of phi = 4 pi G rho, W -> -3/(5-n) G M^2 / R, virial VC -> 0 -> virial sums
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as O
from paper_1602_05700_gb300 import inputs as I


# ---- exact Riemann solution (ideal gas), from the shock and rarefaction wave curves -------------------------

def exact_riemann(wl, wr, gamma, xi):
    """(rho, u, p) at similarity coordinates xi = x / t for left/right states (rho, u, p)."""
    rl, ul, pl = wl
    rr, ur, pr = wr
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)

    def f(p, rk, pk, ak):
        if p > pk:  # shock
            A = 2.0 / ((gamma + 1.0) * rk)
            B = (gamma - 1.0) / (gamma + 1.0) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2.0 * ak / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)

    ps = brentq(lambda p: f(p, rl, pl, al) + f(p, rr, pr, ar) + ur - ul, 1e-12, 100.0 * max(pl, pr), xtol=1e-15)
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, ar) - f(ps, rl, pl, al))
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s < us:  # left of the contact
            if ps > pl:
                sh = ul - al * np.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                out[:, n] = (rl, ul, pl) if s < sh else (rl * (ps / pl + g1) / (g1 * ps / pl + 1), us, ps)
            else:
                ast = al * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s < ul - al:
                    out[:, n] = (rl, ul, pl)
                elif s > us - ast:
                    out[:, n] = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    c = 2 / (gamma + 1) + g1 / al * (ul - s)
                    out[:, n] = (rl * c ** (2 / (gamma - 1)), 2 / (gamma + 1) * (al + (gamma - 1) / 2 * ul + s),
                                 pl * c ** (2 * gamma / (gamma - 1)))
        else:
            if ps > pr:
                sh = ur + ar * np.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                out[:, n] = (rr, ur, pr) if s > sh else (rr * (ps / pr + g1) / (g1 * ps / pr + 1), us, ps)
            else:
                ast = ar * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s > ur + ar:
                    out[:, n] = (rr, ur, pr)
                elif s < us + ast:
                    out[:, n] = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    c = 2 / (gamma + 1) - g1 / ar * (ur - s)
                    out[:, n] = (rr * c ** (2 / (gamma - 1)), 2 / (gamma + 1) * (-ar + (gamma - 1) / 2 * ur + s),
                                 pr * c ** (2 * gamma / (gamma - 1)))
    return out


def test_exact_riemann_helper_on_sod():
    """Textbook star state of Sod's problem (gamma = 1.4): p* = 0.30313, u* = 0.92745."""
    r = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, np.array([0.5, 1.2]))
    assert abs(r[2, 0] - 0.30313) < 1e-5 and abs(r[1, 0] - 0.92745) < 1e-5
    assert abs(r[0, 0] - 0.42632) < 1e-5 and abs(r[0, 1] - 0.26557) < 1e-5


def run_to(hg, U, t_end, cfl=0.3, A=None):
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(cfl * hg.h / O.hydro_max_speed(hg, U), t_end - t)
        O.hydro_step(hg, U, dt, A)
        t += dt
    return U


def sod_run(n, axis, gamma=1.4):
    shape = [1, 1, 1]
    shape[2 - axis] = n
    hg = O.HydroGrid(*shape[::-1], 1.0 / n, gamma)
    U = O.hydro_cons(hg, I.shock_tube(tuple(shape), axis))
    return hg, run_to(hg, U, 0.2)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sod_against_exact_solution_converges(axis):
    errs = []
    for n in (100, 200, 400):
        hg, U = sod_run(n, axis)
        W = O.hydro_prim(hg, U).reshape(5, n)
        x = (np.arange(n) + 0.5) / n - 0.5
        ex = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, x / 0.2)
        errs.append([np.abs(W[0] - ex[0]).mean(), np.abs(W[1 + axis] - ex[1]).mean(), np.abs(W[4] - ex[2]).mean()])
        others = [q for q in (1, 2, 3) if q != 1 + axis]
        assert np.all(W[others] == 0.0)
    errs = np.array(errs)
    assert np.all(errs[0] < [6e-3, 1.2e-2, 4.5e-3]), errs[0]  # MC slopes (minmod: 7.7e-3, 1.5e-2, 6.2e-3)
    # discontinuities limit the L1 rate to about 1 (shock, contact) and 2/3..1 (contact smearing)
    assert np.all(errs[1] < 0.75 * errs[0]) and np.all(errs[2] < 0.75 * errs[1]), errs


def test_one_dimensional_problem_is_identical_along_every_axis():
    fields = []
    for axis in (0, 1, 2):
        hg, U = sod_run(64, axis)
        W = O.hydro_prim(hg, U).reshape(5, 64)
        fields.append((W[0], W[1 + axis], W[4]))
    for f in fields[1:]:
        for a, b in zip(fields[0], f):
            assert np.array_equal(a, b)


# ---- HLLC --------------------------------------------------------------------------------------------------

def physical_flux(w, d, gamma):
    r, v, p = w[0], np.array(w[1:4]), w[4]
    E = p / (gamma - 1) + 0.5 * r * v @ v
    f = np.zeros(5)
    f[0] = r * v[d]
    f[1:4] = r * v[d] * v
    f[1 + d] += p
    f[4] = (E + p) * v[d]
    return f


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency_and_upwinding(d):
    g = 5.0 / 3.0
    w = np.array([1.3, 0.2, -0.4, 0.7, 0.9])
    assert np.allclose(O.hydro_hllc(g, w, w, d), physical_flux(w, d, g), rtol=1e-14, atol=1e-14)
    fast = w.copy()
    fast[1 + d] = 5.0  # supersonic to the right: the flux is the left state's
    other = np.array([0.2, 5.0, 5.0, 5.0, 0.1])
    other[1 + d] = 6.0
    assert np.array_equal(O.hydro_hllc(g, fast, other, d), physical_flux(fast, d, g)) or \
        np.allclose(O.hydro_hllc(g, fast, other, d), physical_flux(fast, d, g), rtol=1e-15, atol=0)
    slow = -fast
    slow[0], slow[4] = fast[0], fast[4]
    other2 = other.copy()
    other2[1 + d] = -6.0
    assert np.allclose(O.hydro_hllc(g, other2, slow, d), physical_flux(slow, d, g), rtol=1e-15, atol=0)


def test_hllc_keeps_an_isolated_stationary_contact():
    n = 64
    hg = O.HydroGrid(n, 1, 1, 1.0 / n, 1.4)
    W = I.shock_tube(hg.shape, 0, left=(1.0, 0.0, 1.0), right=(0.1, 0.0, 1.0))
    U = O.hydro_cons(hg, W)
    U0 = U.copy()
    for _ in range(50):
        O.hydro_step(hg, U, 0.3 * hg.h / O.hydro_max_speed(hg, U))
    assert np.abs(U - U0).max() < 1e-13


# ---- smooth flow, conservation, source terms -----------------------------------------------------------------

def test_smooth_advection_is_second_order():
    errs = []
    for n in (64, 128, 256):
        hg = O.HydroGrid(n, 1, 1, 1.0 / n, 1.4)
        x = (np.arange(n) + 0.5) / n
        W = np.zeros((5, 1, 1, n))
        W[0] = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        W[1] = 1.0
        W[4] = 1.0
        U = run_to(hg, O.hydro_cons(hg, W), 0.1)
        rho = U[0].ravel()
        keep = (x > 0.3) & (x < 0.95)  # away from the inflow edge, whose zero-gradient ghosts are not periodic
        errs.append(np.abs(rho - (1.0 + 0.2 * np.sin(2 * np.pi * (x - 0.1))))[keep].mean())
    assert errs[1] / errs[2] > 3.5 and errs[0] / errs[1] > 3.5, errs


def test_conservation_to_rounding():
    n = 28
    hg = O.HydroGrid(n, n, n, 1.0 / n, 5.0 / 3.0)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = 1.0, 1.0
    W[:, 10:18, 10:18, 10:18] = I.hydro_noise((8, 8, 8), 5)
    U = O.hydro_cons(hg, W)
    tot0 = U.reshape(5, -1).sum(axis=1)
    for _ in range(2):  # each stage reaches 2 cells, so 2 steps do not reach the 10-cell border of gas at rest
        O.hydro_step(hg, U, 0.3 * hg.h / O.hydro_max_speed(hg, U))
    tot = U.reshape(5, -1).sum(axis=1)
    scale = np.abs(U).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot - tot0) <= 1e-14 * scale), (tot - tot0) / scale
    assert np.abs(U[:, :2] - O.hydro_cons(hg, W)[:, :2]).max() == 0.0


def test_strong_blast_stays_positive_and_conservative():
    """A point-like blast (pressure ratio 1e5) in a box of gas at rest: no floor needed, density and pressure stay
    positive, mass and energy are conserved to rounding while the shock is inside the box."""
    n = 24
    hg = O.HydroGrid(n, n, n, 1.0 / n, 1.4)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = 1.0, 1e-5
    W[4, 11:13, 11:13, 11:13] = 1.0
    U = O.hydro_cons(hg, W)
    tot0 = U.reshape(5, -1).sum(axis=1)
    for _ in range(12):
        O.hydro_step(hg, U, 0.3 * hg.h / O.hydro_max_speed(hg, U))
    Wf = O.hydro_prim(hg, U)
    assert np.isfinite(U).all() and Wf[0].min() > 0 and Wf[4].min() > 0
    assert np.abs(U[:, :2] - O.hydro_cons(hg, W)[:, :2]).max() == 0.0  # the shock has not reached the faces
    tot = U.reshape(5, -1).sum(axis=1)
    assert abs(tot[0] - tot0[0]) <= 1e-14 * tot0[0] and abs(tot[4] - tot0[4]) <= 1e-13 * tot0[4]


def test_uniform_field_source_is_exact_heun():
    n = 6
    hg = O.HydroGrid(n, n, n, 1.0 / n, 5.0 / 3.0)
    W = np.zeros((5, n, n, n))
    W[0], W[4] = 1.7, 0.8
    U = O.hydro_cons(hg, W)
    E0 = U[4].copy()
    a = np.array([0.3, -1.1, 0.45])
    A = np.broadcast_to(a[:, None, None, None], (3, n, n, n))
    dt = 0.01
    O.hydro_step(hg, U, dt, A)
    for q in range(3):
        assert np.allclose(U[1 + q], 1.7 * a[q] * dt, rtol=1e-14, atol=0)
    assert np.allclose(U[4] - E0, 0.5 * 1.7 * (a @ a) * dt * dt, rtol=1e-9, atol=0)
    assert np.allclose(U[0], 1.7, rtol=0, atol=0)


def test_characteristic_speed_of_a_hand_computed_state():
    hg = O.HydroGrid(2, 1, 1, 0.5, 5.0 / 3.0)
    W = np.zeros((5, 1, 1, 2))
    W[:, 0, 0, 0] = (1.0, 0.6, 0.8, 0.0, 0.6)   # |v| = 1, a = sqrt(5/3 * 0.6) = 1
    W[:, 0, 0, 1] = (2.0, 0.0, 0.0, 0.3, 1.2)   # |v| = 0.3, a = 1
    assert abs(O.hydro_max_speed(hg, O.hydro_cons(hg, W)) - 2.0) < 1e-15


# ---- polytrope input and virial sums -----------------------------------------------------------------------

def test_lane_emden_closed_forms_and_textbook_constants():
    xs, ts, ds, xi1, om = I.lane_emden(0.0)
    assert abs(xi1 - np.sqrt(6.0)) < 1e-10 and abs(om - 2 * np.sqrt(6.0)) < 1e-9
    assert np.allclose(ts[:-1], 1 - xs[:-1] ** 2 / 6, atol=1e-12)
    xs, ts, ds, xi1, om = I.lane_emden(1.0)
    assert abs(xi1 - np.pi) < 1e-10 and abs(om - np.pi) < 1e-9
    assert np.allclose(ts[1:-1], np.sin(xs[1:-1]) / xs[1:-1], atol=1e-11)
    xs, ts, ds, xi1, om = I.lane_emden(5.0)
    assert np.isnan(xi1)
    assert np.allclose(ts, 1 / np.sqrt(1 + xs ** 2 / 3), atol=1e-10)
    for n, x1, w in ((1.5, 3.65375, 2.71406), (3.0, 6.89685, 2.01824)):  # textbook tables
        _, _, _, xi1, om = I.lane_emden(n)
        assert abs(xi1 - x1) < 1e-5 and abs(om - w) < 1e-5


def test_polytrope_atmosphere_is_hydrostatic_and_dilute():
    """The isothermal atmosphere balances the star's gravity on its own (k_T grad rho_a = -rho_a grad phi, checked
    with central differences along an axis outside the star) and holds a negligible mass."""
    n = 96
    rho0, P0, phi, info0 = I.polytrope(n, atm=0.0)
    rho, P, phi1, info = I.polytrope(n)
    assert np.array_equal(phi, phi1)
    rho_a, p_a = rho - rho0, P - P0
    assert np.allclose(p_a, info["kt"] * rho_a, rtol=1e-12, atol=0)
    c = n // 2
    line = slice(c + n // 3 + 2, n - 2)  # outside the star (R = 1/3) along +x
    h = 1.0 / n
    dpa = (p_a[c, c, line.start + 1:line.stop + 1] - p_a[c, c, line.start - 1:line.stop - 1]) / (2 * h)
    dphi = (phi[c, c, line.start + 1:line.stop + 1] - phi[c, c, line.start - 1:line.stop - 1]) / (2 * h)
    assert np.abs(dpa + rho_a[c, c, line] * dphi).max() < 5e-3 * np.abs(dpa).max()  # central-difference error
    assert 0.0 < info["atm_mass"] < 1e-3
    assert info["rho_atm"] == rho_a.min() > 0.0


def test_polytrope_potential_solves_poisson_and_mass():
    """The exact potential satisfies Poisson's equation: the 7-point Laplacian of its samples matches 4 pi G rho
    with a second-order error."""
    errs = []
    for n in (48, 96):
        rho, P, phi, info = I.polytrope(n, atm=0.0)
        h = 1.0 / n
        lap = (phi[1:-1, 1:-1, 2:] + phi[1:-1, 1:-1, :-2] + phi[1:-1, 2:, 1:-1] + phi[1:-1, :-2, 1:-1]
               + phi[2:, 1:-1, 1:-1] + phi[:-2, 1:-1, 1:-1] - 6 * phi[1:-1, 1:-1, 1:-1]) / h ** 2
        src = 4 * np.pi * rho[1:-1, 1:-1, 1:-1]
        errs.append(np.abs(lap - src).mean() / src.mean())
    assert errs[1] < 5e-3 and errs[0] / errs[1] > 3.5, errs
    assert abs(rho.sum() * h ** 3 - 1.0) < 2e-3
    # hydrostatic balance dP/dr = -rho dphi/dr along the x axis inside the star
    c = n // 2
    line = slice(c, c + n // 4)
    dP = np.gradient(P[c, c, line], h)
    dphi = np.gradient(phi[c, c, line], h)
    assert np.abs(dP[2:-2] + rho[c, c, line][2:-2] * dphi[2:-2]).max() < 2e-2 * np.abs(dP).max()


def test_polytrope_virial_theorem_and_binding_energy():
    W_exact = -1.5  # -3/(5-n) G M^2 / R for n = 3, G = M = 1, R = 1/3 -> -1.5 * 3
    res = []
    for n in (48, 96):
        rho, P, phi, info = I.polytrope(n, atm=0.0)  # the star alone (vacuum cells are not bound)
        hg = O.HydroGrid(n, n, n, 1.0 / n, 5.0 / 3.0)
        Wp = np.zeros((5, n, n, n))
        Wp[0], Wp[4] = rho, P
        v = O.hydro_virial(hg, O.hydro_cons(hg, Wp), phi)
        res.append((abs(v["W"] / (W_exact * 3.0) - 1.0), abs(v["VC"])))
        assert abs(v["K"]) == 0.0
        assert abs(v["M_bound"] - rho.sum() / n ** 3) < 1e-10  # every star cell is bound: all the mass
        assert v["rho_max"] == rho.max()
    # the cell-centre sums of the smooth, compactly supported profile converge far faster than O(h^2): both the
    # binding energy and the virial balance hold to ~1e-10 already at 48^3
    assert all(e < 1e-8 for e, _ in res) and all(vc < 1e-8 for _, vc in res), res
