/*
 * Oracle for the hyperbolic self-gravity scheme (arXiv 1602.05700) -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 C.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library; the product path never does.  It shares no code, header, table or
 * helper with the CUDA library: every formula below is written out here from the paper and from the readings
 * of it that the paper leaves open (those are marked "reading").
 *
 * What is computed (paper Sec. 1, Eq. HNeq.; Sec. 2):
 *   (-1/c^2 d^2/dt^2 + Laplacian) phi = 4 pi G rho
 * stepped explicitly ("simple discretization", Sec. 2).  Reading: cell-centred grid, one ghost layer,
 * 7-point Laplacian, three-level central difference in time (leapfrog):
 *   phi^{n+1} = 2 phi^n - phi^{n-1} + nu^2 * sum_{6 nb}(phi^n_nb - phi^n_c) - (c dt)^2 4 pi G (rho - rho_bar)
 * with nu = c dt / h and rho_bar = 0 except with periodic boundaries (Sec. 4: the mean density is then
 * subtracted from the source).  The neighbour sum is taken in the order -x, +x, -y, +y, -z, +z.
 *
 * Outer boundary conditions (Sec. 2, Sec. 4):
 *   DIRICHLET  ghost values are data.  They come from the multipole expansion of rho (Sec. 4, model aD05):
 *              phi_g = -G sum_{l<=lmax} sum_m 4 pi/(2l+1) Q_lm Y_lm(x_g/r_g) / r_g^{l+1},
 *              Q_lm = sum_j rho_j h^3 r_j^l Y_lm(x_j/r_j), real orthonormal Y_lm, about the coordinate origin.
 *              lmax = 0 is the monopole -G M / r with M = sum rho h^3.
 *   ROBIN      monopole radiation condition (Sec. 2 cites it as a Robin condition equivalent to monopole gravity;
 *              Sec. 4: errors leave through the boundary).  Reading: d_t(r phi) + c d_r(r phi) = 0 with
 *              d_r = d_n / mu, mu = |x_g . n| / r_g, upwinded from the interior neighbour i:
 *              u_g^{n+1} = u_g^n - (nu/mu) (u_g^n - u_i^n),  u = r phi.  Its static limit is r_g phi_g = r_i phi_i.
 *   PERIODIC   ghost = interior cell on the opposite side; source uses rho - mean(rho) (Sec. 4).
 * Only the six face ghost layers are ever read (the 7-point stencil and the central gradient never touch edge
 * or corner ghosts); edge and corner ghost entries are left at zero.
 *
 * Layout: a "ghosted" array has (nz+2)*(ny+2)*(nx+2) doubles, C order (z, y, x), interior cell (i,j,k) at
 * ((k+1)*(ny+2) + (j+1))*(nx+2) + (i+1).  An "interior" array has nz*ny*nx doubles, C order.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define OG_BC_DIRICHLET 0
#define OG_BC_ROBIN 1
#define OG_BC_PERIODIC 2

typedef struct {
    int nx, ny, nz;
    int bc;
    double h;
    double x0, y0, z0; /* lower corner of the domain; cell centres at x0 + (i + 1/2) h */
    double c, G, dt;
} og_grid;

static const double OG_PI = 3.14159265358979323846;

static size_t gidx(const og_grid* g, int i, int j, int k) {
    return ((size_t)(k + 1) * (size_t)(g->ny + 2) + (size_t)(j + 1)) * (size_t)(g->nx + 2) + (size_t)(i + 1);
}
static size_t iidx(const og_grid* g, int i, int j, int k) {
    return ((size_t)k * (size_t)g->ny + (size_t)j) * (size_t)g->nx + (size_t)i;
}
static double cx(const og_grid* g, int i) { return g->x0 + (i + 0.5) * g->h; }
static double cy(const og_grid* g, int j) { return g->y0 + (j + 0.5) * g->h; }
static double cz(const og_grid* g, int k) { return g->z0 + (k + 0.5) * g->h; }
static size_t ncells(const og_grid* g) { return (size_t)g->nx * g->ny * g->nz; }
static size_t nghosted(const og_grid* g) { return (size_t)(g->nx + 2) * (g->ny + 2) * (g->nz + 2); }

/* Whole-array copies and clears.  The library that the tests check is built without OpenMP, where these are plain
 * memcpy / memset and every "omp" line below is ignored.  The benchmark's all-core timing of the oracle builds the
 * same file a second time with -fopenmp: the sweep's z planes and these copies are then split over the host's
 * cores.  Every cell's update reads only the previous levels, so both builds compute the same bits. */
static void copy_array(double* dst, const double* src, size_t n) {
#ifdef _OPENMP
    const size_t chunk = 1 << 16;
#pragma omp parallel for schedule(static)
    for (size_t c = 0; c < (n + chunk - 1) / chunk; ++c) {
        size_t a = c * chunk, m = a + chunk < n ? chunk : n - a;
        memcpy(dst + a, src + a, m * sizeof(double));
    }
#else
    memcpy(dst, src, n * sizeof(double));
#endif
}
static void zero_array(double* dst, size_t n) {
#ifdef _OPENMP
    const size_t chunk = 1 << 16;
#pragma omp parallel for schedule(static)
    for (size_t c = 0; c < (n + chunk - 1) / chunk; ++c) {
        size_t a = c * chunk, m = a + chunk < n ? chunk : n - a;
        memset(dst + a, 0, m * sizeof(double));
    }
#else
    memset(dst, 0, n * sizeof(double));
#endif
}

/* nu = c dt / h ; the source factor (c dt)^2 4 pi G multiplies rho. */
static double og_nu(const og_grid* g) { return g->c * g->dt / g->h; }
static double og_src(const og_grid* g) { return (g->c * g->dt) * (g->c * g->dt) * 4.0 * OG_PI * g->G; }

/* ---- sums -----------------------------------------------------------------------------------------------
 * Reading: a sum the method defines (the multipole moments Q_lm of Sec. 4, the mass, the mean density subtracted
 * from the source with periodic boundaries, Sec. 4) is the exact sum of its terms, rounded once to the nearest
 * double.  That value does not depend on the order of the terms.  A plain running sum of the 1.7e7 cells of a
 * 256^3 grid instead carries a rounding error of order 1e-12 relative, and the lossless scheme carries every bit
 * of the Dirichlet data into phi.
 * The exact sum is held as a nonoverlapping expansion (Shewchuk 1997, "Adaptive precision floating-point
 * arithmetic and fast robust geometric predicates", Grow-Expansion with zero elimination): components in
 * increasing magnitude whose exact sum is the sum of all terms so far; a new term passes through every component
 * by an error-free two-sum, keeping the nonzero rounding errors.  A double expansion has at most a few dozen
 * nonzero components. */
#define OG_XMAX 80
typedef struct {
    int n;
    double p[OG_XMAX];
} og_xsum;

static void xsum_init(og_xsum* s) { s->n = 0; }

static void xsum_add(og_xsum* s, double x) {
    int kept = 0;
    for (int c = 0; c < s->n; ++c) {
        double y = s->p[c];
        double big = fabs(x) >= fabs(y) ? x : y, small = fabs(x) >= fabs(y) ? y : x;
        double t = big + small;
        double err = small - (t - big); /* exact: t + err = x + y */
        if (err != 0.0) s->p[kept++] = err;
        x = t;
    }
    s->p[kept++] = x;
    s->n = kept;
}

/* The expansion's exact value rounded to the nearest double (ties to even).  Walking down from the largest
 * component, t is the rounded sum of the components seen so far and err its exact rounding error; the first
 * nonzero err ends the walk, since every component left is smaller than half an ulp of t.  Those components only
 * matter when err is exactly half an ulp (a tie that the addition broke to even): if they push the same way as
 * err, the exact value lies beyond the midpoint and rounds to t + 2 err. */
static double xsum_value(const og_xsum* s) {
    if (s->n == 0) return 0.0;
    int c = s->n - 1;
    double t = s->p[c], err = 0.0;
    while (c > 0) {
        double y = s->p[--c];
        double u = t + y;
        err = y - (u - t);
        t = u;
        if (err != 0.0) break;
    }
    if (c > 0 && err != 0.0 && ((err > 0.0) == (s->p[c - 1] > 0.0)) && s->p[c - 1] != 0.0) {
        double twice = 2.0 * err;
        double v = t + twice;
        if (v - t == twice) t = v; /* err was exactly half an ulp of t */
    }
    return t;
}

/* exported for the tests: the correctly rounded sum of n doubles */
double og_exact_sum(const double* x, size_t n) {
    og_xsum s;
    xsum_init(&s);
    for (size_t q = 0; q < n; ++q) xsum_add(&s, x[q]);
    return xsum_value(&s);
}

/* mean density (periodic boundaries subtract it from the source, Sec. 4) */
double og_mean(const og_grid* g, const double* rho) { return og_exact_sum(rho, ncells(g)) / (double)ncells(g); }

/* total mass sum rho h^3 */
double og_mass(const og_grid* g, const double* rho) {
    return og_exact_sum(rho, ncells(g)) * g->h * g->h * g->h;
}

/* ---- face iteration: face f in 0..5 = (-x, +x, -y, +y, -z, +z) ------------------------------------------- */
/* For face f and in-face indices (a, b), give the ghost cell (gi,gj,gk) and its interior neighbour (ii,ij,ik). */
static void face_cells(const og_grid* g, int f, int a, int b, int* gc, int* ic) {
    int axis = f / 2, hi = f % 2;
    int n[3] = {g->nx, g->ny, g->nz};
    int cell[3];
    /* the two in-face axes, in increasing order */
    int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
    cell[t0] = a;
    cell[t1] = b;
    cell[axis] = hi ? n[axis] : -1;
    gc[0] = cell[0]; gc[1] = cell[1]; gc[2] = cell[2];
    cell[axis] = hi ? n[axis] - 1 : 0;
    ic[0] = cell[0]; ic[1] = cell[1]; ic[2] = cell[2];
}
static void face_extent(const og_grid* g, int f, int* na, int* nb) {
    int axis = f / 2;
    int n[3] = {g->nx, g->ny, g->nz};
    int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
    *na = n[t0];
    *nb = n[t1];
}

/* ---- real orthonormal spherical harmonics --------------------------------------------------------------- */
/* Y_lm at the direction (x,y,z)/r, r > 0, for 0 <= l <= lmax, stored at l*l + l + m.  Associated Legendre
 * functions by the standard upward recurrences in l (with the Condon-Shortley phase), then
 * Y_l0 = K_l0 P_l^0, Y_lm = sqrt2 K_lm P_l^m cos(m phi), Y_l,-m = sqrt2 K_lm P_l^m sin(m phi), m > 0,
 * K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). */
static void real_ylm(int lmax, double x, double y, double z, double* Y) {
    double r = sqrt(x * x + y * y + z * z);
    double ct = z / r;
    double st = sqrt(x * x + y * y) / r;
    double ph = atan2(y, x);
    double P[32][32]; /* P[l][m], lmax <= 31 */
    for (int m = 0; m <= lmax; ++m) {
        double pmm = 1.0;
        for (int q = 1; q <= m; ++q) pmm *= -(2.0 * q - 1.0) * st;
        P[m][m] = pmm;
        if (m + 1 <= lmax) P[m + 1][m] = ct * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= lmax; ++l)
            P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
    }
    for (int l = 0; l <= lmax; ++l) {
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0; /* (l-m)!/(l+m)! */
            for (int q = l - m + 1; q <= l + m; ++q) ratio /= (double)q;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * OG_PI) * ratio);
            if (m == 0) {
                Y[l * l + l] = K * P[l][0];
            } else {
                Y[l * l + l + m] = sqrt(2.0) * K * P[l][m] * cos(m * ph);
                Y[l * l + l - m] = sqrt(2.0) * K * P[l][m] * sin(m * ph);
            }
        }
    }
}

/* exported for the tests (addition-theorem pin) */
void og_real_ylm(int lmax, double x, double y, double z, double* Y) { real_ylm(lmax, x, y, z, Y); }

/* Multipole moments Q_lm = sum_j rho_j h^3 r_j^l Y_lm(x_j / r_j) about the coordinate origin (Sec. 4, Dirichlet
 * boundary by multipole expansion), each the exact sum of its terms rounded once (see "sums" above).  Q has
 * (lmax+1)^2 entries.  A cell centred exactly at the origin adds only to
 * Q_00 (r^l Y_lm vanishes there for l > 0). */
void og_moments(const og_grid* g, const double* rho, int lmax, double* Q) {
    int nq = (lmax + 1) * (lmax + 1);
    double Y[32 * 32];
    double h3 = g->h * g->h * g->h;
    og_xsum* acc = (og_xsum*)malloc((size_t)nq * sizeof(og_xsum));
    for (int q = 0; q < nq; ++q) xsum_init(&acc[q]);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double m = rho[iidx(g, i, j, k)] * h3;
                double x = cx(g, i), y = cy(g, j), z = cz(g, k);
                double r = sqrt(x * x + y * y + z * z);
                if (r == 0.0) {
                    xsum_add(&acc[0], m / sqrt(4.0 * OG_PI));
                    continue;
                }
                real_ylm(lmax, x, y, z, Y);
                double rl = 1.0;
                for (int l = 0; l <= lmax; ++l) {
                    for (int mm = -l; mm <= l; ++mm) xsum_add(&acc[l * l + l + mm], m * rl * Y[l * l + l + mm]);
                    rl *= r;
                }
            }
    for (int q = 0; q < nq; ++q) Q[q] = xsum_value(&acc[q]);
    free(acc);
}

/* Exterior multipole potential at (x,y,z): -G sum_l 4 pi/(2l+1) r^{-(l+1)} sum_m Q_lm Y_lm. */
double og_multipole_phi(const og_grid* g, int lmax, const double* Q, double x, double y, double z) {
    double Y[32 * 32];
    double r = sqrt(x * x + y * y + z * z);
    real_ylm(lmax, x, y, z, Y);
    double phi = 0.0;
    double rinv = 1.0 / r, rp = rinv;
    for (int l = 0; l <= lmax; ++l) {
        double s = 0.0;
        for (int m = -l; m <= l; ++m) s += Q[l * l + l + m] * Y[l * l + l + m];
        phi += 4.0 * OG_PI / (2.0 * l + 1.0) * s * rp;
        rp *= rinv;
    }
    return -g->G * phi;
}

/* Fill the six face ghost layers of phi with the multipole potential. */
void og_fill_multipole_ghosts(const og_grid* g, int lmax, const double* Q, double* phi) {
    for (int f = 0; f < 6; ++f) {
        int na, nb;
        face_extent(g, f, &na, &nb);
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int gc[3], ic[3];
                face_cells(g, f, a, b, gc, ic);
                phi[gidx(g, gc[0], gc[1], gc[2])] = og_multipole_phi(g, lmax, Q, cx(g, gc[0]), cy(g, gc[1]), cz(g, gc[2]));
            }
    }
}

/* Periodic ghosts: each face ghost is the interior cell on the opposite side. */
void og_fill_periodic_ghosts(const og_grid* g, double* phi) {
    int n[3] = {g->nx, g->ny, g->nz};
    for (int f = 0; f < 6; ++f) {
        int na, nb;
        face_extent(g, f, &na, &nb);
        int axis = f / 2, hi = f % 2;
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int gc[3], ic[3];
                face_cells(g, f, a, b, gc, ic);
                int src[3] = {gc[0], gc[1], gc[2]};
                src[axis] = hi ? 0 : n[axis] - 1;
                phi[gidx(g, gc[0], gc[1], gc[2])] = phi[gidx(g, src[0], src[1], src[2])];
            }
    }
}

/* Robin ghosts at their static limit r_g phi_g = r_i phi_i (used when a state is seeded). */
void og_fill_robin_static_ghosts(const og_grid* g, double* phi) {
    for (int f = 0; f < 6; ++f) {
        int na, nb;
        face_extent(g, f, &na, &nb);
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int gc[3], ic[3];
                face_cells(g, f, a, b, gc, ic);
                double xg = cx(g, gc[0]), yg = cy(g, gc[1]), zg = cz(g, gc[2]);
                double xi = cx(g, ic[0]), yi = cy(g, ic[1]), zi = cz(g, ic[2]);
                double rg = sqrt(xg * xg + yg * yg + zg * zg), ri = sqrt(xi * xi + yi * yi + zi * zi);
                phi[gidx(g, gc[0], gc[1], gc[2])] = phi[gidx(g, ic[0], ic[1], ic[2])] * ri / rg;
            }
    }
}

/* Robin coefficient of a face ghost: nu/mu with mu = |x_g . n| / r_g. */
static double robin_coef(const og_grid* g, int f, const int* gc) {
    double xg = cx(g, gc[0]), yg = cy(g, gc[1]), zg = cz(g, gc[2]);
    double rg = sqrt(xg * xg + yg * yg + zg * zg);
    double along = f / 2 == 0 ? xg : (f / 2 == 1 ? yg : zg);
    double mu = fabs(along) / rg;
    return og_nu(g) / mu;
}

/* Laplacian numerator sum_{6 nb}(phi_nb - phi_c) in the order -x, +x, -y, +y, -z, +z. */
static double nb_sum(const og_grid* g, const double* phi, int i, int j, int k) {
    double c = phi[gidx(g, i, j, k)];
    double s = 0.0;
    s += phi[gidx(g, i - 1, j, k)] - c;
    s += phi[gidx(g, i + 1, j, k)] - c;
    s += phi[gidx(g, i, j - 1, k)] - c;
    s += phi[gidx(g, i, j + 1, k)] - c;
    s += phi[gidx(g, i, j, k - 1)] - c;
    s += phi[gidx(g, i, j, k + 1)] - c;
    return s;
}

/* One sub-step of Eq. HNeq.: phi_next from phi (level n, with valid ghosts) and phi_prev (level n-1, interior).
 * Writes the interior and the face ghosts of phi_next. */
void og_step(const og_grid* g, const double* phi, const double* phi_prev, const double* rho, double* phi_next) {
    double nu = og_nu(g);
    double nu2 = nu * nu;
    double src = og_src(g);
    double rho_bar = g->bc == OG_BC_PERIODIC ? og_mean(g, rho) : 0.0;
    zero_array(phi_next, nghosted(g));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = gidx(g, i, j, k);
                double L = nb_sum(g, phi, i, j, k);
                phi_next[q] = 2.0 * phi[q] - phi_prev[q] + nu2 * L - src * (rho[iidx(g, i, j, k)] - rho_bar);
            }
    if (g->bc == OG_BC_PERIODIC) {
        og_fill_periodic_ghosts(g, phi_next);
        return;
    }
    for (int f = 0; f < 6; ++f) {
        int na, nb;
        face_extent(g, f, &na, &nb);
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int gc[3], ic[3];
                face_cells(g, f, a, b, gc, ic);
                size_t qg = gidx(g, gc[0], gc[1], gc[2]);
                if (g->bc == OG_BC_DIRICHLET) {
                    phi_next[qg] = phi[qg]; /* boundary data, frozen while rho is frozen (Sec. 2) */
                } else {
                    double xg = cx(g, gc[0]), yg = cy(g, gc[1]), zg = cz(g, gc[2]);
                    double xi = cx(g, ic[0]), yi = cy(g, ic[1]), zi = cz(g, ic[2]);
                    double rg = sqrt(xg * xg + yg * yg + zg * zg), ri = sqrt(xi * xi + yi * yi + zi * zi);
                    double ug = rg * phi[qg], ui = ri * phi[gidx(g, ic[0], ic[1], ic[2])];
                    double ug_next = ug - robin_coef(g, f, gc) * (ug - ui);
                    phi_next[qg] = ug_next / rg;
                }
            }
    }
}

/* n sub-steps.  phi (level n) and phi_prev (level n-1) are ghosted arrays and are advanced in place:
 * on return they hold levels n+nsteps and n+nsteps-1.  work is a ghosted scratch array. */
void og_run(const og_grid* g, double* phi, double* phi_prev, const double* rho, int nsteps, double* work) {
    size_t n = nghosted(g);
    for (int s = 0; s < nsteps; ++s) {
        og_step(g, phi, phi_prev, rho, work);
        copy_array(phi_prev, phi, n);
        copy_array(phi, work, n);
    }
}

/* Gravitational acceleration -grad phi by second-order central differences (ghosts supply the face values). */
void og_accel(const og_grid* g, const double* phi, double* ax, double* ay, double* az) {
    double inv2h = 1.0 / (2.0 * g->h);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = iidx(g, i, j, k);
                ax[q] = -(phi[gidx(g, i + 1, j, k)] - phi[gidx(g, i - 1, j, k)]) * inv2h;
                ay[q] = -(phi[gidx(g, i, j + 1, k)] - phi[gidx(g, i, j - 1, k)]) * inv2h;
                az[q] = -(phi[gidx(g, i, j, k + 1)] - phi[gidx(g, i, j, k - 1)]) * inv2h;
            }
}

/* Steady-state residual r = Laplacian_h phi - 4 pi G (rho - rho_bar) over the interior.
 * out[0] = root mean square of r, out[1] = max |r|. */
void og_residual(const og_grid* g, const double* phi, const double* rho, double* out) {
    double rho_bar = g->bc == OG_BC_PERIODIC ? og_mean(g, rho) : 0.0;
    double ih2 = 1.0 / (g->h * g->h);
    double s2 = 0.0, mx = 0.0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double r = nb_sum(g, phi, i, j, k) * ih2 - 4.0 * OG_PI * g->G * (rho[iidx(g, i, j, k)] - rho_bar);
                s2 += r * r;
                if (fabs(r) > mx) mx = fabs(r);
            }
    out[0] = sqrt(s2 / (double)ncells(g));
    out[1] = mx;
}

/* Interior norms of a and b (ghosted): out[0] = ||a-b||_2 / ||b||_2, out[1] = max|a-b| / max|b|,
 * out[2] = the paper's average relative error <dphi~> = sqrt(mean(((a-b)/b)^2)) (Sec. 4, Eq. error; a = phi_H,
 * b = phi_P, uniform cells so the volume weights cancel). */
void og_compare(const og_grid* g, const double* a, const double* b, double* out) {
    double d2 = 0.0, b2 = 0.0, dm = 0.0, bm = 0.0, e2 = 0.0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = gidx(g, i, j, k);
                double d = a[q] - b[q];
                d2 += d * d;
                b2 += b[q] * b[q];
                if (fabs(d) > dm) dm = fabs(d);
                if (fabs(b[q]) > bm) bm = fabs(b[q]);
                e2 += (d / b[q]) * (d / b[q]);
            }
    out[0] = sqrt(d2 / b2);
    out[1] = dm / bm;
    out[2] = sqrt(e2 / (double)ncells(g));
}

/* ---- discrete adjoint ------------------------------------------------------------------------------------
 * The T sub-steps map rho linearly (plus a rho-independent part from the initial state and Dirichlet data) to
 * phi^T.  Given lam_T = dL/dphi^T on the interior, return dL/drho by transposing each sub-step in reverse
 * order.  The forward states are not needed: the recursion is linear.  Dirichlet ghosts are data (the
 * dependence of multipole ghosts on rho is not differentiated), Robin ghosts are state, periodic ghosts are
 * copies of the interior. */
static void adjoint_substep(const og_grid* g, double* lam_next, double* lam_cur, double* lam_prev, double* grad) {
    int n[3] = {g->nx, g->ny, g->nz};
    double nu = og_nu(g), nu2 = nu * nu, src = og_src(g);
    /* transpose of the ghost update of level n+1 */
    for (int f = 0; f < 6; ++f) {
        int na, nb;
        face_extent(g, f, &na, &nb);
        int axis = f / 2, hi = f % 2;
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                int gc[3], ic[3];
                face_cells(g, f, a, b, gc, ic);
                size_t qg = gidx(g, gc[0], gc[1], gc[2]);
                double lg = lam_next[qg];
                lam_next[qg] = 0.0;
                if (g->bc == OG_BC_PERIODIC) {
                    int src_c[3] = {gc[0], gc[1], gc[2]};
                    src_c[axis] = hi ? 0 : n[axis] - 1;
                    lam_next[gidx(g, src_c[0], src_c[1], src_c[2])] += lg;
                } else if (g->bc == OG_BC_ROBIN) {
                    double xg = cx(g, gc[0]), yg = cy(g, gc[1]), zg = cz(g, gc[2]);
                    double xi = cx(g, ic[0]), yi = cy(g, ic[1]), zi = cz(g, ic[2]);
                    double rg = sqrt(xg * xg + yg * yg + zg * zg), ri = sqrt(xi * xi + yi * yi + zi * zi);
                    double a_ = robin_coef(g, f, gc);
                    lam_cur[qg] += (1.0 - a_) * lg;
                    lam_cur[gidx(g, ic[0], ic[1], ic[2])] += a_ * ri / rg * lg;
                }
            }
    }
    /* transpose of the interior update */
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t q = gidx(g, i, j, k);
                double l = lam_next[q];
                lam_cur[q] += 2.0 * l - 6.0 * nu2 * l;
                lam_cur[gidx(g, i - 1, j, k)] += nu2 * l;
                lam_cur[gidx(g, i + 1, j, k)] += nu2 * l;
                lam_cur[gidx(g, i, j - 1, k)] += nu2 * l;
                lam_cur[gidx(g, i, j + 1, k)] += nu2 * l;
                lam_cur[gidx(g, i, j, k - 1)] += nu2 * l;
                lam_cur[gidx(g, i, j, k + 1)] += nu2 * l;
                lam_prev[q] -= l;
                grad[iidx(g, i, j, k)] -= src * l;
            }
    if (g->bc == OG_BC_DIRICHLET) {
        /* adjoint mass that reached Dirichlet ghosts is dropped: those values are data */
        for (int f = 0; f < 6; ++f) {
            int na, nb;
            face_extent(g, f, &na, &nb);
            for (int b = 0; b < nb; ++b)
                for (int a = 0; a < na; ++a) {
                    int gc[3], ic[3];
                    face_cells(g, f, a, b, gc, ic);
                    lam_cur[gidx(g, gc[0], gc[1], gc[2])] = 0.0;
                }
        }
    }
}

void og_adjoint(const og_grid* g, const double* lam_T, int T, double* grad) {
    size_t n = nghosted(g), nc = ncells(g);
    double* a = (double*)calloc(n, sizeof(double));
    double* b = (double*)calloc(n, sizeof(double));
    double* c = (double*)calloc(n, sizeof(double));
    double *lam_next = a, *lam_cur = b, *lam_prev = c;
    for (size_t q = 0; q < nc; ++q) grad[q] = 0.0;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) lam_next[gidx(g, i, j, k)] = lam_T[iidx(g, i, j, k)];
    for (int s = T - 1; s >= 0; --s) {
        adjoint_substep(g, lam_next, lam_cur, lam_prev, grad);
        double* t = lam_next;
        lam_next = lam_cur;
        lam_cur = lam_prev;
        lam_prev = t;
        memset(lam_prev, 0, n * sizeof(double));
    }
    if (g->bc == OG_BC_PERIODIC) {
        /* transpose of rho -> rho - mean(rho) */
        double m = og_mean(g, grad);
        for (size_t q = 0; q < nc; ++q) grad[q] -= m;
    }
    free(a);
    free(b);
    free(c);
}
