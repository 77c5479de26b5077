/*
 * hg.h -- C ABI of the GB300 (sm_103a) hyperbolic self-gravity library.
 *
 * The library advances the wave-equation replacement of Poisson's equation (arXiv 1602.05700, Sec. 1,
 * Eq. HNeq.)
 *
 *     (-1/c_h^2 d^2/dt^2 + Laplacian) phi = 4 pi G rho
 *
 * by explicit sub-steps on a uniform Cartesian grid (Sec. 2: "simple discretization", wave sub-steps on their own
 * time-line with rho frozen, c_h = k_g (c_s + |v|) chosen by the caller), with the outer boundary conditions of
 * Sec. 2 and Sec. 4 (Robin / monopole radiation, Dirichlet by multipole expansion, periodic with the mean density
 * removed), and returns the gravitational acceleration -grad phi that a hydro code consumes.
 *
 * Discretisation (the paper leaves it open; this is the library's reading):
 *   cell-centred cells of side h, cell (i,j,k) centred at origin + (i+1/2, j+1/2, k+1/2) h, one ghost layer;
 *   nu = c_h dt / h;
 *   phi^{n+1} = 2 phi^n - phi^{n-1} + nu^2 sum_{6 nb}(phi^n_nb - phi^n) - (c_h dt)^2 4 pi G (rho - rho_bar),
 *   rho_bar = mean(rho) with periodic boundaries, else 0; phi^0 = phi^{-1} = 0 unless seeded.
 *   Stable for nu sqrt(3) <= 1 (checked by hg_init_grid).
 *
 * Conventions for every entry point:
 *   - Return value: HG_OK (0) or a negative HG_ERR_* code; hg_last_error() then gives a message (thread-local).
 *     No call aborts, traps or waits without bound: every wait inside a kernel has a time limit (1 s), after which
 *     the kernel records the failure in the grid's device error word and returns; hg_sync and hg_get_stats then
 *     report HG_ERR_TIMEOUT.
 *   - Debug builds (the library compiled with -DHG_DEBUG) also check, before every global store of the sub-step
 *     kernels, that the padded index range lies inside its array; a range outside is not stored and sets a second
 *     bit of the error word, which hg_sync and hg_get_stats report as HG_ERR_BOUNDS.  Release builds carry no checks.
 *   - Array arguments are plain pointers.  Unless stated otherwise an array is nz*ny*nx elements in C order
 *     (z slowest, x fastest), no padding, of the element type given by a dtype argument (HG_DT_F32 = float,
 *     HG_DT_F64 = double).  A flag *_on_device says whether a pointer is device memory of the grid's device
 *     (1) or host memory (0).  The caller owns every pointer it passes; the library copies what it keeps.
 *   - All device work is enqueued on the CUDA stream given to hg_init_grid.  Calls that return data to host
 *     memory synchronise that stream; hg_step and the device-to-device calls do not.
 *   - A grid is used from one host thread at a time.
 */
#ifndef HG_H
#define HG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HG_OK 0
#define HG_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, unknown enum, ...) */
#define HG_ERR_CFL (-2)       /* time step violates nu sqrt(3) <= 1, or the Robin boundary's nu/mu <= 1 */
#define HG_ERR_CUDA (-3)      /* a CUDA runtime call failed; the message names it */
#define HG_ERR_NONFINITE (-4) /* a NaN or Inf was found in the state (hg_get_stats) */
#define HG_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define HG_ERR_STATE (-6)     /* call not valid in the grid's current state */
#define HG_ERR_BOUNDS (-7)    /* debug builds: a sub-step kernel computed a store index outside its array */

/* storage / arithmetic precision of a grid's state */
#define HG_PREC_F32K 0 /* float storage, compensated (Kahan-style) increments of phi */
#define HG_PREC_F64 1  /* double storage and arithmetic: the reference mode */

/* element type of caller buffers */
#define HG_DT_F32 0
#define HG_DT_F64 1

/* outer boundary conditions (Sec. 2 and Sec. 4) */
#define HG_BC_DIRICHLET_ANALYTIC 0  /* ghost phi = -G M / r, M = sum rho h^3 (monopole of the density) */
#define HG_BC_DIRICHLET_MULTIPOLE 1 /* ghost phi from the multipole expansion of rho up to l = lmax */
#define HG_BC_ROBIN 2               /* monopole radiation condition d_t(r phi) + c_h d_r(r phi) = 0 */
#define HG_BC_PERIODIC 3            /* wrap-around; the source uses rho - mean(rho) */

#define HG_MAX_LMAX 8

typedef struct hg_grid hg_grid;

/* FP64 diagnostics of the current state (Sec. 4, Eq. error, and the steady-state check of Eq. Poissoneq.). */
typedef struct {
    double mass;           /* sum rho h^3 over the interior (as stored) */
    double residual_rms;   /* rms over the interior of Laplacian_h phi^n - 4 pi G (rho - rho_bar) */
    double residual_max;   /* max of |...| */
    double change_rel;     /* ||phi^n - phi^{n-1}||_2 / ||phi^n||_2 over the interior */
    double phi_max;        /* max |phi^n| over the interior */
    long long step;        /* sub-steps taken since the last hg_set_phi / hg_init_grid */
    int nonfinite;         /* 1 if a NaN or Inf was seen in phi^n, phi^{n-1} or rho */
} hg_stats;

/*
 * Create a grid of nx*ny*nz cells of side h whose lower corner is origin[3] (so cell centres are at
 * origin + (idx + 1/2) h).  c_h is the gravity wave speed (Sec. 2: c_g = k_g (c_s + |v|)), G the gravitational
 * constant, dt the sub-step.  precision is HG_PREC_*, bc is HG_BC_*, lmax the multipole order for
 * HG_BC_DIRICHLET_MULTIPOLE (0..HG_MAX_LMAX; ignored otherwise).  cuda_stream is a cudaStream_t (NULL = the
 * legacy default stream) on the current device; all later work of this grid goes there.
 * phi^0 = phi^{-1} = 0 and rho = 0 on return.  Errors: HG_ERR_ARG (sizes < 1, h/c_h/dt <= 0, bad enum),
 * HG_ERR_CFL (nu sqrt(3) > 1; for Robin also any ghost with nu/mu > 1, i.e. the domain must surround the
 * origin), HG_ERR_CUDA (allocation).  On error *g is NULL.
 */
int hg_init_grid(hg_grid** g, int nx, int ny, int nz, double h, const double origin[3], double c_h, double G,
                 double dt, int precision, int bc, int lmax, void* cuda_stream);

/*
 * Set the density (Sec. 2: rho is frozen during the wave sub-steps of one hydro step).  rho: nz*ny*nx values of
 * type dtype, host or device.  Recomputes the FP64 mass, the mean (periodic) and, for the Dirichlet modes, the
 * FP64 multipole moments and the ghost values of phi^n and phi^{n-1} (Sec. 4, Dirichlet boundary by multipole
 * expansion).  The interior of phi is not touched.  With a device density the call does not wait for the GPU
 * (except in the Dirichlet modes, whose moments come back to the host): the mass and mean are read back lazily
 * by the next call that reports them (hg_get_stats, hg_save_state), and rho must stay valid until the grid's
 * stream has run the work.  With a host density the call returns after the copy has been consumed.
 */
int hg_set_density(hg_grid* g, const void* rho, int dtype, int on_device);

/*
 * Seed the state: phi^n = phi, phi^{n-1} = phi_prev (phi_prev may be NULL: then phi^{n-1} = phi^n, i.e. zero
 * initial time derivative).  Sec. 2 seeds phi from a Poisson solve.  Ghosts are set per boundary condition:
 * Dirichlet data, periodic copies, or the Robin static limit r_g phi_g = r_i phi_i.  Resets the step count.
 */
int hg_set_phi(hg_grid* g, const void* phi, const void* phi_prev, int dtype, int on_device);

/* Advance n_substeps >= 0 sub-steps.  Asynchronous on the grid's stream. */
int hg_step(hg_grid* g, int n_substeps);

/*
 * Number of sub-steps fused per pass over the grid in hg_step: 1 = one sweep per sub-step (default); k in
 * 2..HG_MAX_TEMPORAL_DEPTH advances k sub-steps per round trip through HBM (rho is frozen across them, Sec. 2).
 * HG_ERR_ARG for k out of range or for an FP64 grid, HG_ERR_STATE for a slab (hg_init_slab).  The inner levels of a
 * fused pass never reach memory: by default they keep the compensation of phi as a float, which is a little more
 * accurate than the 16-bit code of a stored level, and the results differ from k single sweeps by rounding (a
 * changed compensation can flip the rounding of a later increment), both staying within the compensated scheme's
 * accuracy against FP64.  With hg_set_temporal_exact(g, 1) the inner levels round their compensation as a store and a
 * load would, and the results are bit-identical to k single sweeps, at some cost in speed (measured at k = 2, 512^3,
 * Robin: 0.424 ms per sub-step by default, 0.519 exact, 0.503 for single sweeps).  k = 2 on Dirichlet and Robin grids
 * runs a TMA-staged kernel; other depths and periodic grids a generic one (slower than single sweeps).
 */
#define HG_MAX_TEMPORAL_DEPTH 8
int hg_set_temporal_depth(hg_grid* g, int k);
int hg_set_temporal_exact(hg_grid* g, int exact);

/* z planes per thread block of the single-sweep kernel (a tuning knob: more blocks and more z warm-up below, fewer
 * and longer blocks above); 0 restores the built-in rule.  Results do not depend on it. */
int hg_set_block_depth(hg_grid* g, int planes);

/*
 * Gravitational acceleration a = -grad phi^n by second-order central differences, ghosts supplying the face
 * values.  ax, ay, az: device buffers of nz*ny*nx elements of type dtype.  Asynchronous.
 */
int hg_accel(hg_grid* g, void* ax, void* ay, void* az, int dtype);

/* Copy phi^n (interior) into out: nz*ny*nx elements of type dtype, host or device.  For HG_PREC_F32K with
 * dtype HG_DT_F64 the compensated value (float + its compensation, summed in double) is returned. */
int hg_get_phi(hg_grid* g, void* out, int dtype, int on_device);

/* Copy phi^n including its face ghosts into out: (nz+2)*(ny+2)*(nx+2) doubles in host memory, C order,
 * interior cell (i,j,k) at ((k+1)(ny+2) + j+1)(nx+2) + i+1; edge and corner entries are 0. */
int hg_get_phi_ghosted(hg_grid* g, double* out);

/* FP64 diagnostics of the current state (synchronises the stream).  Returns HG_ERR_NONFINITE (with *s filled)
 * when a NaN or Inf is present. */
int hg_get_stats(hg_grid* g, hg_stats* s);

/* The FP64 multipole moments Q_lm = sum rho h^3 r^l Y_lm (real orthonormal Y_lm about the coordinate origin),
 * (lmax+1)^2 doubles at index l*l + l + m, of the last hg_set_density (HG_ERR_STATE unless a Dirichlet mode). */
int hg_get_moments(hg_grid* g, double* Q);

/*
 * Compare phi^n with a reference potential phi_P (Sec. 4, Eq. error): out[0] = ||phi - phi_P||_2 / ||phi_P||_2,
 * out[1] = max|phi - phi_P| / max|phi_P|, out[2] = the paper's average relative error
 * sqrt(mean(((phi - phi_P) / phi_P)^2)).  phi_P: nz*ny*nx doubles, host or device.
 */
int hg_compare(hg_grid* g, const double* phi_P, int on_device, double out[3]);

/* Checkpoint / resume of the full state (bit-exact): hg_state_bytes gives the size of the opaque buffer that
 * hg_save_state fills and hg_load_state reads, in host memory (on_device = 0) or device memory (on_device = 1).
 * A buffer is only valid for a grid of the same sizes, precision, boundary condition and lmax, and with
 * bit-identical h, origin, c_h, G and dt (the stored source, the Dirichlet data and the Robin coefficients depend on
 * them); hg_load_state returns HG_ERR_ARG, and changes nothing, for any other buffer. */
size_t hg_state_bytes(const hg_grid* g);
int hg_save_state(hg_grid* g, void* buf, int on_device);
int hg_load_state(hg_grid* g, const void* buf, int on_device);

/*
 * Adjoint of the sub-stepping: dL/drho for a loss L of the potentials phi^m produced by hg_step from a fixed initial
 * state (the paper has no adjoint; this is the transpose of the discretised Eq. HNeq.).  The sub-step is linear, so
 * the reverse recursion needs no forward state:
 *   hg_adjoint_reset(g)                   lambda = 0, running sum = 0 (the first call allocates a shadow state);
 *   hg_adjoint_inject(g, dL/dphi^m, ...)  adds the direct derivative of L with respect to phi^m (interior cells,
 *                                         nz*ny*nx values) at the current reverse level m;
 *   hg_adjoint_step(g, n)                 n reverse sub-steps (m -> m - n), adding each level's lambda to the sum;
 *   hg_adjoint_grad(g, out, ...)          out = dL/drho = -(c_h dt)^2 4 pi G sum_m lambda^m (minus its mean for
 *                                         periodic boundaries), nz*ny*nx values.
 * For L = L(phi^T) after T forward sub-steps: reset, inject(dL/dphi^T), step(T), grad.  For losses on several
 * levels, inject each dL/dphi^m when the reverse sweep reaches m.  Dirichlet boundary data are treated as constants
 * (their dependence on rho through the multipole moments is not differentiated); Robin ghosts and periodic copies
 * are part of the state and are transposed exactly.  The adjoint state has the precision of the grid.
 */
int hg_adjoint_reset(hg_grid* g);
int hg_adjoint_inject(hg_grid* g, const void* dL_dphi, int dtype, int on_device);
int hg_adjoint_step(hg_grid* g, int n_substeps);
int hg_adjoint_grad(hg_grid* g, void* dL_drho, int dtype, int on_device);
/* The whole terminal-loss case in one call: dL_drho = dL/drho for L = L(phi^T) after T forward sub-steps, given
 * dL_dphiT = dL/dphi^T (both nz*ny*nx values of element type dtype, on the device if on_device); the same as reset,
 * inject, step(T), grad.  No checkpoint interval is taken: the reverse recursion of the linear sub-step needs no
 * forward state (checkpointing matters for losses on intermediate potentials and is done by the Python binding's
 * autograd.trajectory_loss).  HG_ERR_ARG for T < 0 or null pointers. */
int hg_adjoint(hg_grid* g, const void* dL_dphiT, int T, void* dL_drho, int dtype, int on_device);

/*
 * Measurement hooks.  hg_profile(g, 1) makes the library record a pair of CUDA events on the grid's stream around
 * every launch of its sub-step kernel (the single-sweep or the temporally blocked stencil); hg_profile(g, 0) stops.
 * hg_profile_read synchronises the stream and returns the summed duration (ms) and the number of those timed
 * launches since the previous read (then resets both), and the total number of kernels the library has launched
 * for this grid since its creation.  Any output pointer may be NULL.
 */
int hg_profile(hg_grid* g, int enable);
int hg_profile_read(hg_grid* g, double* substep_kernel_ms, long long* substep_launches, long long* kernel_launches);

/*
 * One hydro step's gravity with host input and output, pipelined across calls (Sec. 2: rho frozen over the
 * sub-steps of a hydro step, -grad phi handed back to the hydro code).  Enqueues, without waiting for the GPU:
 *   the copy of rho_host (nz*ny*nx values of rho_dtype) to a device slot on an upload stream of the grid,
 *   hg_set_density from that slot, n_substeps sub-steps (hg_step), -grad phi (hg_accel, central differences) into
 *   a device slot, and its copy to ax_host, ay_host, az_host (nz*ny*nx values of acc_dtype each) on a download
 *   stream of the grid.
 * Two device slots alternate, and the grid's stream waits only on the upload it consumes; a slot is refilled only
 * after its previous contents have been used (ordered by events, not by the host).  With two calls in flight
 * (hg_io_wait(g, 2) after each call) the upload of call s+1 and the download of call s-1 both run under the
 * sub-steps of call s.  rho_host may be NULL (the source is unchanged) and the three acceleration pointers
 * may all be NULL (no output).  The host buffers must be page-locked for the copies to overlap (pageable memory
 * works, synchronously) and belong to the library until hg_io_wait has covered the call.  Device memory: two
 * density slots and two acceleration slots, allocated on first use.  Errors: HG_ERR_ARG (bad dtype, only some
 * acceleration pointers), HG_ERR_CUDA.
 */
int hg_io_step(hg_grid* g, const void* rho_host, int rho_dtype, int n_substeps, void* ax_host, void* ay_host,
               void* az_host, int acc_dtype);

/* Block until all but the newest `keep` hg_io_step calls have finished (their host buffers are then the caller's
 * again and the accelerations are in place).  keep = 0 waits for every call. */
int hg_io_wait(hg_grid* g, int keep);

/*
 * Diagnostic of the bounded waits inside the kernels: launches a one-block kernel that waits (1 ms limit) on an
 * mbarrier nothing will complete, then reads the grid's device error word as hg_sync does.  Returns HG_OK when the
 * wait gave up and the timeout was reported (the error word is cleared again), HG_ERR_STATE when it was not, or the
 * error of an earlier launch if one was pending.  Synchronises the stream.
 */
int hg_check_bounded_wait(hg_grid* g);

/*
 * Diagnostic of the debug build's index checks: launches a one-thread kernel that passes the index one past the
 * grid's padded array (never stored) to the same check the sub-step kernels use, then reads the error word as hg_sync
 * does.  Returns HG_OK when the check fired and HG_ERR_BOUNDS was reported (the error word is cleared again),
 * HG_ERR_STATE when it was not, the error of an earlier launch if one was pending, and HG_ERR_STATE without launching
 * anything in a release build.  hg_is_debug_build() tells which build is loaded (1 debug, 0 release).
 */
int hg_check_bounds(hg_grid* g);
int hg_is_debug_build(void);

/* Block until the grid's streams are idle; HG_ERR_CUDA carries any pending asynchronous error. */
int hg_sync(hg_grid* g);

/* Release the grid and its device memory (NULL is allowed). */
void hg_free(hg_grid* g);

/*
 * Batches: many independent grids (any sizes, both precisions, any boundary conditions) advanced together.  Every
 * sub-step of all grids is one batched kernel launch (plus one batched ghost-copy launch if some grid is periodic);
 * hg_batch_step records its n sub-steps once as a CUDA graph and replays it with one graph launch, on a stream of
 * the batch that is ordered after, and before, the grids' own stream.  Results are bit-identical to hg_step on each
 * grid (single sweeps: the grids' temporal depth is not used here).  The first hg_batch_step autotunes the z extent
 * of a block by timing its first sub-steps (all candidates compute the same result) and caches the choice per
 * device and set of grid shapes for the process.  All grids must live on one device and share one stream; a grid
 * may belong to several batches and may also be stepped on its own between batch steps.
 */
typedef struct hg_batch hg_batch;
int hg_batch_create(hg_grid* const* grids, int n, hg_batch** b);
int hg_batch_step(hg_batch* b, int n_substeps);
/* autotuned FP64 z planes per block (0 before the first hg_batch_step) and blocks per batched sub-step launch */
int hg_batch_info(const hg_batch* b, int* z_planes_per_block, long long* blocks_per_substep);
/* the whole autotuned launch: out[0] = FP64 z planes per block, out[1] = FP64 tile rows (0: per grid, 128- or
 * 32-cell rows, whichever leaves fewer lanes idle; 4: 128-cell rows for every grid), out[2] = compensated-float
 * (TMA-staged) z planes per block, out[3] = 1 when the two precisions run as separate launches per sub-step (two
 * independent chains on two streams; 0: one launch holds both).  The choice is timed on the first sub-steps of the
 * first hg_batch_step and cached per device and set of grids for the life of the process (an autotuner of this
 * library; the paper has no counterpart). */
int hg_batch_tuning(const hg_batch* b, int out[4]);
/* Pin the launch mode instead of letting the autotuner choose it: mode 1 = split (one launch per precision class per
 * sub-step, two streams), 0 = one launch for both, -1 = autotuned (the default).  The other knobs are still tuned, on
 * the next hg_batch_step; results do not depend on any of them.  HG_ERR_ARG for another mode. */
int hg_batch_set_split(hg_batch* b, int mode);
void hg_batch_free(hg_batch* b);

/*
 * The FP64 multipole moments Q_lm of a density, computed without allocating any GPU memory.
 *
 * The paper has no counterpart to this call; it exists for callers that are not allowed to call cudaMalloc: code
 * whose device memory is owned and budgeted by someone else (a framework's caching allocator, a fixed-size pool
 * shared by several solvers), or a loop that must not take the device-wide synchronisation a cudaMalloc or
 * cudaFree can imply.  Such a caller cannot create a grid (hg_init_grid allocates its state), but can still get
 * the boundary moments of its own density: it passes the input and the output, and the library supplies the
 * scratch.
 *
 * rho: nz*ny*nx values of type dtype in device memory (C order, x fastest), cell (i,j,k) centred at
 * origin + (i+1/2, j+1/2, k+1/2) h.  Q: (lmax+1)^2 doubles, in device memory (Q_on_device = 1) or host memory
 * (Q_on_device = 0: the call then synchronises the stream); same definition and index as hg_get_moments.
 * cuda_stream: the stream the work is enqueued on (NULL = legacy default stream), on the current device.
 *
 * Scratch: a fixed array compiled into the library, 2 x 152 x 81 + 81 doubles (197,640 bytes), present on every GPU
 * that loads the library until the process exits.  Its size is what bounds lmax: lmax > HG_MAX_LMAX is rejected
 * with HG_ERR_ARG; grid sizes are not limited by it.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and caches it; make that first call before any stream
 * capture.  The cache is keyed by the device and its CUDA context, so after a cudaDeviceReset the next call looks
 * the address up again (in the new context) instead of using the old one.  All calls on a device share the one array: every call overwrites the partial sums it uses, so no
 * state carries over from the previous call, but calls whose GPU work overlaps in time (other streams, other host
 * threads) race on the array and must be serialised by the caller.
 * Errors: HG_ERR_ARG (null pointer, bad dtype, sizes < 1, h <= 0, lmax out of range), HG_ERR_CUDA.
 */
int hg_moments_noalloc(const void* rho, int dtype, int nx, int ny, int nz, double h, const double origin[3], int lmax,
                       double* Q, int Q_on_device, void* cuda_stream);

/*
 * Slab decomposition of one grid along z.  The paper notes that the method needs only communication between
 * neighbouring cells, which suits distributed memory (Sec. 4, timing discussion; Sec. 5).  A grid of nz planes is
 * split into slabs of consecutive planes, each an hg_grid of its own (origin shifted by k0 h along z, same h, c_h,
 * G, dt, precision, boundary condition), one per device or process.  Before every sub-step each slab's interface
 * ghost planes must hold the neighbouring slabs' boundary planes of phi^n:
 *   hg_init_slab(..., z_interfaces)    hg_init_grid for a slab: bit 0 / bit 1 of z_interfaces make the -z / +z face an
 *                                      interface (the other faces keep the boundary condition; an interface face
 *                                      needs no boundary data and is exempt from the Robin stability and geometry
 *                                      checks).  Robin and Dirichlet boundaries only (HG_ERR_STATE for periodic),
 *                                      temporal depth 1 only (the exchange is per sub-step), no batches, no adjoint.
 *   hg_set_z_interface(g, lo, hi)      the same flags on an existing grid (its faces have passed the checks).
 *   hg_plane_bytes(g)                  size of one packed plane: nx*ny doubles (F64), or nx*ny floats followed by nx*ny
 *                                      16-bit compensation codes (F32K).
 *   hg_get_plane(g, which, buf, dev)   copies the first (which = 0, k = 0) or last (which = 1, k = nz-1) interior
 *                                      plane of phi^n into buf (device memory if dev, else host; host copies return
 *                                      after the copy, device copies are ordered on the grid's stream).
 *   hg_put_ghost_plane(g, side, buf, dev)  copies a packed plane into the -z (side 0) or +z (side 1) ghost plane of
 *                                      phi^n; HG_ERR_STATE unless that face is an interface.
 *   hg_set_boundary_moments(g, Q)      Dirichlet modes: evaluates the face ghosts (both time levels) from given
 *                                      moments Q ((lmax+1)^2 doubles, host memory) -- the sum over all slabs of their
 *                                      own moments (hg_get_moments after hg_set_density), so that every slab's outer
 *                                      faces see the expansion of the whole density.
 * With these, k sub-steps of the slabs (exchange, then hg_step(g, 1) on every slab, k times) reproduce k sub-steps of
 * the whole grid bit for bit (Robin; Dirichlet up to the rounding of the summed moments).
 */
int hg_init_slab(hg_grid** g, int nx, int ny, int nz, double h, const double origin[3], double c_h, double G,
                 double dt, int precision, int bc, int lmax, void* cuda_stream, int z_interfaces);
int hg_set_z_interface(hg_grid* g, int lo, int hi);
size_t hg_plane_bytes(const hg_grid* g);
int hg_get_plane(hg_grid* g, int which, void* buf, int on_device);
int hg_put_ghost_plane(hg_grid* g, int side, const void* buf, int on_device);
int hg_set_boundary_moments(hg_grid* g, const double* Q);

/*
 * Measured arithmetic rate of the current GPU (a measurement aid for the rooflines of pipe-bound kernels; the paper
 * has no counterpart): kind 0 = FP64 fused multiply-add, 1 = FP32 fused multiply-add, 2 = the packed FP32 pair
 * (two multiply-adds in one instruction).  Independent dependency chains on 8 blocks of 256 threads per SM, best of
 * five event-timed launches after a warm-up.  instr_per_s: thread-level instructions per second; ops_per_s
 * (may be NULL): multiply-adds per second.  Synchronous (its own stream).  Errors: HG_ERR_ARG, HG_ERR_CUDA.
 */
int hg_probe_rate(int kind, double* instr_per_s, double* ops_per_s);

/* Message of the last failing call on this host thread ("" if none). */
const char* hg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HG_H */
