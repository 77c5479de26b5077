/*
 * Oracle for the hydrodynamics that consumes the hyperbolic gravity (arXiv 1602.05700) -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 C, loaded only by the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark.  It shares no code with the CUDA library; every formula is written out here from the paper's
 * description of its host code and from the readings listed below.
 *
 * Paper Sec. 2: ideal-gas hydrodynamics (gamma = 5/3) by a finite-volume method with an HLLC-type approximate
 * Riemann solver (the paper's HLLD solver without magnetic field), Cartesian coordinates in 3D, outgoing outer
 * boundaries; self-gravity enters the momentum and energy equations through -grad phi, with phi from the wave
 * equation advanced k_g times per hydro step while rho is held fixed.
 *
 * Readings (the paper names the solver family only):
 *   state        conserved u = (rho, rho vx, rho vy, rho vz, E), E = P/(gamma-1) + rho |v|^2 / 2.
 *   reconstruction  piecewise linear in the primitives w = (rho, vx, vy, vz, P) with monotonized-central
 *                limited slopes, mc(a, b) = the argument of least magnitude among 2a, (a + b)/2, 2b when all
 *                three have one sign, else 0:
 *                left state at face s+1/2  w_s + mc(w_s - w_{s-1}, w_{s+1} - w_s) / 2,
 *                right state               w_{s+1} - mc(w_{s+1} - w_s, w_{s+2} - w_{s+1}) / 2.
 *                (A minmod limiter, the more diffusive choice, flattens the peaked core of the paper's n = 3
 *                star: its central density would fall by 6.5% in ~4 dynamical times at the paper's resolution,
 *                where Sec. 3 reports a decline of about 2% in ~5.)
 *   Riemann      HLLC (Toro, Spruce & Speares 1994) with Davis' wave-speed bounds
 *                S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R), a = sqrt(gamma P / rho).
 *   boundary     outgoing = zero gradient: the two ghost layers repeat the edge cell (indices clamped).
 *   time         two-stage SSP Runge-Kutta (Heun): u1 = u0 + dt L(u0), u2 = (u0 + (u1 + dt L(u1))) / 2, with
 *                L(u) = -div F / h + S(u) and S = (0, rho a, m . a) for the acceleration a = -grad phi, which is
 *                held fixed over the hydro step (phi after the step's wave sub-steps).
 *   floors       after each stage: rho < rho_floor -> rho_floor; P < P_floor -> E = P_floor/(gamma-1) + kinetic.
 *   virial       the paper's VC = (W + 3 (gamma-1) U) / |W| over bound cells (E + rho phi < 0), W = h^3/2 sum rho
 *                phi, U = h^3 sum (E - kinetic).
 * No fused multiply-add: the library is built with -ffp-contract=off.
 *
 * Layout: a field set is 5 planes of nz*ny*nx doubles ("structure of arrays"), plane q at q*n, cell (i,j,k) at
 * (k*ny + j)*nx + i; an acceleration is 3 such planes (ax, ay, az).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double h, gamma, rho_floor, p_floor;
} oh_grid;

static size_t oh_n(const oh_grid* g) { return (size_t)g->nx * g->ny * g->nz; }

/* cell index with the outgoing (zero-gradient) boundary: out-of-range indices are clamped to the edge cell */
static size_t cidx(const oh_grid* g, int i, int j, int k) {
    if (i < 0) i = 0;
    if (i > g->nx - 1) i = g->nx - 1;
    if (j < 0) j = 0;
    if (j > g->ny - 1) j = g->ny - 1;
    if (k < 0) k = 0;
    if (k > g->nz - 1) k = g->nz - 1;
    return ((size_t)k * g->ny + j) * g->nx + i;
}

static void load_cons(const oh_grid* g, const double* U, size_t c, double u[5]) {
    const size_t n = oh_n(g);
    for (int q = 0; q < 5; ++q) u[q] = U[q * n + c];
}

/* kinetic energy density from the conserved state */
static double kinetic(const double u[5], double* vx, double* vy, double* vz) {
    *vx = u[1] / u[0];
    *vy = u[2] / u[0];
    *vz = u[3] / u[0];
    return 0.5 * ((u[1] * *vx + u[2] * *vy) + u[3] * *vz);
}

static void cons_to_prim(double gm1, const double u[5], double w[5]) {
    double vx, vy, vz;
    const double ke = kinetic(u, &vx, &vy, &vz);
    w[0] = u[0];
    w[1] = vx;
    w[2] = vy;
    w[3] = vz;
    w[4] = gm1 * (u[4] - ke);
}

/* conserved state of a primitive state: E = P/(gamma-1) + (rho/2)|v|^2 */
static void prim_to_cons(double gm1, const double w[5], double u[5]) {
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = w[4] / gm1 + 0.5 * w[0] * ((w[1] * w[1] + w[2] * w[2]) + w[3] * w[3]);
}

void oh_cons_from_prim(const oh_grid* g, const double* W, double* U) {
    const size_t n = oh_n(g);
    const double gm1 = g->gamma - 1.0;
    for (size_t c = 0; c < n; ++c) {
        double w[5], u[5];
        for (int q = 0; q < 5; ++q) w[q] = W[q * n + c];
        prim_to_cons(gm1, w, u);
        for (int q = 0; q < 5; ++q) U[q * n + c] = u[q];
    }
}

void oh_prim_from_cons(const oh_grid* g, const double* U, double* W) {
    const size_t n = oh_n(g);
    const double gm1 = g->gamma - 1.0;
    for (size_t c = 0; c < n; ++c) {
        double w[5], u[5];
        load_cons(g, U, c, u);
        cons_to_prim(gm1, u, w);
        for (int q = 0; q < 5; ++q) W[q * n + c] = w[q];
    }
}

/* monotonized-central slope from the one-sided differences a (backward) and b (forward) */
static double mc(double a, double b) {
    const double c = 0.5 * (a + b), a2 = 2.0 * a, b2 = 2.0 * b;
    if (a > 0.0 && b > 0.0) {
        double m = c;
        if (a2 < m) m = a2;
        if (b2 < m) m = b2;
        return m;
    }
    if (a < 0.0 && b < 0.0) {
        double m = c;
        if (a2 > m) m = a2;
        if (b2 > m) m = b2;
        return m;
    }
    return 0.0;
}

/* conserved state u and physical flux f along axis d of the primitive state w */
static void state_flux(double gm1, const double w[5], int d, double u[5], double f[5]) {
    prim_to_cons(gm1, w, u);
    const double un = w[1 + d];
    const double mf = w[0] * un;
    f[0] = mf;
    f[1] = mf * w[1];
    f[2] = mf * w[2];
    f[3] = mf * w[3];
    f[1 + d] = f[1 + d] + w[4];
    f[4] = (u[4] + w[4]) * un;
}

/* HLLC flux along axis d between the primitive states wl (left) and wr (right) */
void oh_hllc(double gamma, const double wl[5], const double wr[5], int d, double F[5]) {
    const double gm1 = gamma - 1.0;
    double ul[5], fl[5], ur[5], fr[5];
    state_flux(gm1, wl, d, ul, fl);
    state_flux(gm1, wr, d, ur, fr);
    const double al = sqrt(gamma * wl[4] / wl[0]);
    const double ar = sqrt(gamma * wr[4] / wr[0]);
    const double unl = wl[1 + d], unr = wr[1 + d];
    const double a1 = unl - al, a2 = unr - ar, b1 = unl + al, b2 = unr + ar;
    const double sl = a1 < a2 ? a1 : a2;
    const double sr = b1 > b2 ? b1 : b2;
    if (sl >= 0.0) {
        memcpy(F, fl, sizeof(fl));
        return;
    }
    if (sr <= 0.0) {
        memcpy(F, fr, sizeof(fr));
        return;
    }
    const double dl = wl[0] * (sl - unl);
    const double dr = wr[0] * (sr - unr);
    const double ss = ((wr[4] - wl[4]) + (unl * dl - unr * dr)) / (dl - dr); /* contact speed S* */
    const int left = ss >= 0.0;
    const double* w = left ? wl : wr;
    const double* u = left ? ul : ur;
    const double* f = left ? fl : fr;
    const double sk = left ? sl : sr;
    const double dk = left ? dl : dr;
    const double unk = w[1 + d];
    const double fac = dk / (sk - ss);
    double us[5];
    us[0] = fac;
    us[1] = fac * w[1];
    us[2] = fac * w[2];
    us[3] = fac * w[3];
    us[1 + d] = fac * ss;
    us[4] = fac * (u[4] / w[0] + (ss - unk) * (ss + w[4] / dk));
    for (int q = 0; q < 5; ++q) F[q] = f[q] + sk * (us[q] - u[q]);
}

/* primitive state of the cell at offset t along axis d from cell (i,j,k) */
static void prim_at(const oh_grid* g, const double* U, int i, int j, int k, int d, int t, double w[5]) {
    double u[5];
    if (d == 0) i += t;
    else if (d == 1) j += t;
    else k += t;
    load_cons(g, U, cidx(g, i, j, k), u);
    cons_to_prim(g->gamma - 1.0, u, w);
}

/* flux through the face between offsets t and t+1 along axis d from cell (i,j,k) */
static void face_flux(const oh_grid* g, const double* U, int i, int j, int k, int d, int t, double F[5]) {
    double wm[5], w0[5], wp[5], wpp[5], wl[5], wr[5];
    prim_at(g, U, i, j, k, d, t - 1, wm);
    prim_at(g, U, i, j, k, d, t, w0);
    prim_at(g, U, i, j, k, d, t + 1, wp);
    prim_at(g, U, i, j, k, d, t + 2, wpp);
    for (int q = 0; q < 5; ++q) {
        wl[q] = w0[q] + 0.5 * mc(w0[q] - wm[q], wp[q] - w0[q]);
        wr[q] = wp[q] - 0.5 * mc(wp[q] - w0[q], wpp[q] - wp[q]);
    }
    oh_hllc(g->gamma, wl, wr, d, F);
}

/* L(u) = -div F / h + S(u) for every cell; A (3 planes) or NULL for no gravity */
void oh_residual(const oh_grid* g, const double* U, const double* A, double* L) {
    const size_t n = oh_n(g);
    const double inv_h = 1.0 / g->h;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double r[5], lo[5], hi[5];
                for (int d = 0; d < 3; ++d) {
                    face_flux(g, U, i, j, k, d, -1, lo);
                    face_flux(g, U, i, j, k, d, 0, hi);
                    for (int q = 0; q < 5; ++q) r[q] = d == 0 ? lo[q] - hi[q] : r[q] + (lo[q] - hi[q]);
                }
                const size_t c = cidx(g, i, j, k);
                for (int q = 0; q < 5; ++q) r[q] = r[q] * inv_h;
                if (A) {
                    double u[5];
                    load_cons(g, U, c, u);
                    const double ax = A[c], ay = A[n + c], az = A[2 * n + c];
                    r[1] = r[1] + u[0] * ax;
                    r[2] = r[2] + u[0] * ay;
                    r[3] = r[3] + u[0] * az;
                    r[4] = r[4] + ((u[1] * ax + u[2] * ay) + u[3] * az);
                }
                for (int q = 0; q < 5; ++q) L[q * n + c] = r[q];
            }
}

static void apply_floors(const oh_grid* g, double u[5]) {
    if (u[0] < g->rho_floor) u[0] = g->rho_floor;
    double vx, vy, vz;
    const double ke = kinetic(u, &vx, &vy, &vz);
    const double gm1 = g->gamma - 1.0;
    const double p = gm1 * (u[4] - ke);
    if (p < g->p_floor) u[4] = g->p_floor / gm1 + ke;
}

/* one hydro step of dt in place; work holds 10 planes (the stage-1 state and a residual) */
void oh_step(const oh_grid* g, double* U, const double* A, double dt, double* work) {
    const size_t n = oh_n(g);
    double* U1 = work;
    double* L = work + 5 * n;
    oh_residual(g, U, A, L);
    for (size_t c = 0; c < n; ++c) {
        double u[5];
        for (int q = 0; q < 5; ++q) u[q] = U[q * n + c] + dt * L[q * n + c];
        apply_floors(g, u);
        for (int q = 0; q < 5; ++q) U1[q * n + c] = u[q];
    }
    oh_residual(g, U1, A, L);
    for (size_t c = 0; c < n; ++c) {
        double u[5];
        for (int q = 0; q < 5; ++q) u[q] = 0.5 * (U[q * n + c] + (U1[q * n + c] + dt * L[q * n + c]));
        apply_floors(g, u);
        for (int q = 0; q < 5; ++q) U[q * n + c] = u[q];
    }
}

/* max over cells of |v| + a, the characteristic speed of the paper's c_g = k_g (c_s + |v|) */
double oh_max_speed(const oh_grid* g, const double* U) {
    const size_t n = oh_n(g);
    const double gm1 = g->gamma - 1.0;
    double m = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double u[5], w[5];
        load_cons(g, U, c, u);
        cons_to_prim(gm1, u, w);
        const double s = sqrt((w[1] * w[1] + w[2] * w[2]) + w[3] * w[3]) + sqrt(g->gamma * w[4] / w[0]);
        if (s > m) m = s;
    }
    return m;
}

/* out = {W, U, K, VC, rho_max, M_bound} over the bound cells (E + rho phi < 0); phi is an interior array */
void oh_virial(const oh_grid* g, const double* U, const double* phi, double* out) {
    const size_t n = oh_n(g);
    double srp = 0.0, su = 0.0, sk = 0.0, sm = 0.0, rmax = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double u[5], vx, vy, vz;
        load_cons(g, U, c, u);
        if (u[0] > rmax) rmax = u[0];
        const double rp = u[0] * phi[c];
        if (u[4] + rp < 0.0) {
            const double ke = kinetic(u, &vx, &vy, &vz);
            srp += rp;
            su += u[4] - ke;
            sk += ke;
            sm += u[0];
        }
    }
    const double h3 = g->h * g->h * g->h;
    const double W = 0.5 * srp * h3;
    const double Ui = su * h3;
    out[0] = W;
    out[1] = Ui;
    out[2] = sk * h3;
    out[3] = (W + 3.0 * (g->gamma - 1.0) * Ui) / fabs(W);
    out[4] = rmax;
    out[5] = sm * h3;
}
