/*
 * hg_hydro.h -- C ABI of the ideal-gas hydrodynamics that consumes the hyperbolic self-gravity of hg.h.
 *
 * The paper (arXiv 1602.05700, Sec. 2) couples its wave-equation gravity to a finite-volume hydro code: ideal gas
 * with gamma = 5/3, an HLLC-type approximate Riemann solver (its HLLD solver with the magnetic field off),
 * Cartesian coordinates in 3D, outgoing outer boundaries, and the wave equation advanced k_g times per hydro step
 * with rho frozen.  It checks the coupling by the virial measure VC = (W + 3 (gamma - 1) U) / |W| of a polytrope
 * (Sec. 3, Eq. VC).  This library provides that host code in its minimal form, so the whole coupled step runs on
 * the GPU:
 *
 *   state        conserved u = (rho, rho vx, rho vy, rho vz, E), E = P/(gamma-1) + rho |v|^2 / 2, on the same
 *                nx*ny*nz cells as the gravity grid;
 *   fluxes       piecewise-linear primitives (rho, v, P) with monotonized-central limited slopes (the
 *                least-magnitude of 2a, (a+b)/2, 2b for one-sided differences a, b of one sign, else 0), HLLC
 *                fluxes with Davis' wave-speed bounds, faces of all three axes in one unsplit update;
 *   boundary     outgoing (zero gradient: two ghost layers repeat the edge cell);
 *   time         two-stage SSP Runge-Kutta (Heun), each stage L(u) = -div F / h + (0, rho a, m . a);
 *   gravity      a = -grad phi of the wave solution after the step's k_g sub-steps, held over the hydro step;
 *   floors       after each stage rho >= rho_floor, P >= p_floor (E raised, momentum kept).
 * These choices are the library's reading: the paper names the solver family only.
 *
 * Conventions are those of hg.h (status codes, hg_last_error, dtype codes, *_on_device flags, caller-owned
 * pointers).  A field set is 5 planes of nz*ny*nx values in C order (z slowest), plane q at offset q*nz*ny*nx:
 * conserved (rho, mx, my, mz, E) or primitive (rho, vx, vy, vz, P).  All device work goes to the stream given to
 * hg_hydro_init; a coupled step requires the gravity grid to use the same stream.
 */
#ifndef HG_HYDRO_H
#define HG_HYDRO_H

#include "hg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hg_hydro hg_hydro;

/* Create the hydro state on the current CUDA device: nx*ny*nz cells of side h, adiabatic index gamma > 1, floors
 * rho_floor >= 0 and p_floor >= 0, state precision dtype (HG_DT_F32: float storage and arithmetic, HG_DT_F64:
 * double, the reference mode that reproduces the CPU oracle's operation order), stream cuda_stream (a
 * cudaStream_t, NULL = legacy default).  The state starts at zero; set it before stepping.  HG_ERR_ARG for bad
 * sizes or parameters, HG_ERR_CUDA if an allocation fails (nothing is leaked). */
int hg_hydro_init(hg_hydro** out, int nx, int ny, int nz, double h, double gamma, double rho_floor, double p_floor,
                  int dtype, void* cuda_stream);

/* Set the state from primitive fields W (5 planes: rho, vx, vy, vz, P) of element type dtype (either), converted
 * to conserved variables on the device in the state's precision.  Host input is copied before the call returns. */
int hg_hydro_set_primitive(hg_hydro* H, const void* W, int dtype, int on_device);

/* Set / read the conserved state (5 planes) in the state's own element type (dtype must match it).  Reading to
 * host memory synchronises the stream. */
int hg_hydro_set_state(hg_hydro* H, const void* U, int dtype, int on_device);
int hg_hydro_get_state(hg_hydro* H, void* U, int dtype, int on_device);

/* max over cells of |v| + sqrt(gamma P / rho): the characteristic speed of the hydro CFL condition and of the
 * paper's c_g = k_g (c_s + |v|) (Sec. 2).  Synchronises the stream. */
int hg_hydro_max_speed(hg_hydro* H, double* s);

/* One coupled hydro step (Sec. 2), asynchronous on the stream:
 *   g != NULL: rho of the current state becomes g's density (hg_set_density semantics: source, mass, and for
 *              the Dirichlet modes the moments and boundary data), g advances n_substeps wave sub-steps, and
 *              a = -grad phi is taken from the advanced potential;
 *   then the two Runge-Kutta stages of length dt with that a (g == NULL: no gravity; n_substeps ignored).
 * g must have the same nx, ny, nz and stream.  HG_ERR_ARG for dt <= 0, n_substeps < 0 or a mismatched grid. */
int hg_hydro_step(hg_hydro* H, hg_grid* g, double dt, int n_substeps);

/* Virial measure of the paper's Eq. VC over the bound cells (E + rho phi < 0), with phi the current potential
 * of g (same nx, ny, nz and stream): out = {W, U, K, VC, rho_max, M_bound} with W = h^3/2 sum rho phi,
 * U = h^3 sum (E - rho |v|^2 / 2), K = h^3 sum rho |v|^2 / 2, VC = (W + 3 (gamma-1) U) / |W|, rho_max over all
 * cells, M_bound = h^3 sum rho.  FP64 sums in a fixed order (deterministic).  Synchronises the stream. */
int hg_hydro_virial(hg_hydro* H, hg_grid* g, double out[6]);

/* Kernel launches made by this hydro state so far (the coupled step's gravity launches are counted by g). */
int hg_hydro_launches(hg_hydro* H, long long* n);

/* Measurement of the Runge-Kutta stage kernel: while enabled, CUDA events on the stream bracket every stage launch.
 * hg_hydro_profile_read synchronises the stream, returns the summed event time (ms) and the number of stage launches
 * since the last read, and resets both.  Disabling keeps what was recorded until the next read. */
int hg_hydro_profile(hg_hydro* H, int enable);
int hg_hydro_profile_read(hg_hydro* H, double* stage_ms, long long* stage_launches);

void hg_hydro_free(hg_hydro* H);

#ifdef __cplusplus
}
#endif

#endif /* HG_HYDRO_H */
