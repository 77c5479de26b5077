// Internal definitions shared by the translation units of the CUDA library (not part of the C ABI).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hg.h"

namespace hg {

// An NVTX range around every ABI call, so that a profiler's timeline shows which call enqueued which kernels (a
// push and a pop of a named range; without an attached tool both return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define HG_RANGE(name) ::hg::NvtxRange hg_nvtx_range_(name)

// Debug builds (-DHG_DEBUG; builder.build(debug=True) makes _build/libhypergrav_debug.so, loaded when the environment
// sets HG_DEBUG=1): before each global store of the sub-step kernels the padded index range is checked against the
// array; a range outside sets bit value 2 of the grid's error word (reported as HG_ERR_BOUNDS) and the store is
// skipped -- no trap, no fault.  Release builds compile the check to `true`.
#ifdef HG_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
__device__ __forceinline__ bool idx_ok(long long q, int n, long long size, int* err) {
    if constexpr (kDebugChecks) {
        if (q < 0 || q + n > size) {
            if (err) atomicOr(err, 2);
            return false;
        }
    }
    return true;
}


// ---- device memory layout ------------------------------------------------------------------------------------
// Every per-cell field of a grid lives in one "padded" array of pitch * (ny+2) * (nz+2) elements: z-planes of
// (ny+2) rows of `pitch` elements.  Row index j+1 and plane index k+1 hold interior cell (i,j,k); the ghost rows
// and planes are j = -1, ny and k = -1, nz.  Inside a row the interior starts at element `xoff` (16 bytes), so the
// x ghosts sit at xoff-1 and xoff+nx and every 4-cell group starting at a multiple of 4 is one aligned 16-byte
// (float4 / 2 x double2) access.  The pitch is a multiple of 128 bytes and leaves room for a full vector read of
// the last group of a row.
struct Layout {
    int nx, ny, nz;
    int xoff;      // elements before interior x = 0 in a row
    long long pitch;  // elements per row
    long long plane;  // elements per z-plane = pitch * (ny + 2)
    long long elems;  // total elements = plane * (nz + 2)
    __host__ __device__ long long at(int i, int j, int k) const {
        return (long long)(k + 1) * plane + (long long)(j + 1) * pitch + xoff + i;
    }
};

inline Layout make_layout(int nx, int ny, int nz, int esize) {
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.xoff = 16 / esize;
    int align = 128 / esize;
    long long need = (long long)L.xoff + nx + 4;
    L.pitch = (need + align - 1) / align * align;
    L.plane = L.pitch * (ny + 2);
    L.elems = L.plane * (nz + 2);
    return L;
}

// ---- face ghosts -----------------------------------------------------------------------------------------------
// Faces f = 0..5 are -x, +x, -y, +y, -z, +z.  Face f has na x nb ghost cells; x faces are indexed (a,b) = (j,k),
// y faces (i,k), z faces (i,j).  Ghosts of all faces are enumerated face after face, a fastest.
struct Faces {
    long long off[7];
    int na[6], nb[6];
};

inline Faces make_faces(int nx, int ny, int nz) {
    Faces F;
    int n[3] = {nx, ny, nz};
    F.off[0] = 0;
    for (int f = 0; f < 6; ++f) {
        int axis = f / 2;
        int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
        F.na[f] = n[t0];
        F.nb[f] = n[t1];
        F.off[f + 1] = F.off[f] + (long long)F.na[f] * F.nb[f];
    }
    return F;
}

// ghost cell (g) and interior neighbour (in) of face ghost number t; returns the face
__host__ __device__ inline int face_cell(const Faces& F, int nx, int ny, int nz, long long t, int g[3], int in[3]) {
    int f = 0;
    while (f < 5 && t >= F.off[f + 1]) ++f;
    long long r = t - F.off[f];
    int a = (int)(r % F.na[f]), b = (int)(r / F.na[f]);
    int axis = f / 2, hi = f % 2;
    int n[3] = {nx, ny, nz};
    int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
    g[t0] = a;
    g[t1] = b;
    g[axis] = hi ? n[axis] : -1;
    in[0] = g[0];
    in[1] = g[1];
    in[2] = g[2];
    in[axis] = hi ? n[axis] - 1 : 0;
    return f;
}

// ---- multipole constants -----------------------------------------------------------------------------------------
constexpr int kMaxL = HG_MAX_LMAX;
constexpr int kMaxQ = (kMaxL + 1) * (kMaxL + 1);
struct YlmNorm {
    double n[kMaxQ];        // normalisation of r^l Y_lm written as n_lm * q_l^m(z, r^2) * {C_m, S_m}
    double inv_lm[kMaxQ];   // 1 / (l - m) for the upward recurrence (index l*l + l + m, m >= 0)
};
void fill_ylm_norms(YlmNorm& N);

// storage unit of the compensation of a compensated-float state (a 16-bit code, decoded in cell.cuh)
typedef unsigned short lo_code;

// ---- the grid --------------------------------------------------------------------------------------------------
}  // namespace hg

struct hg_grid {
    int nx, ny, nz;
    double h;
    double origin[3];
    double c, G, dt;
    int prec, bc, lmax;
    cudaStream_t stream;
    int device;
    double nu, nu2, src;  // nu = c dt / h, nu^2, (c dt)^2 4 pi G
    int esize;
    hg::Layout L;
    hg::Faces F;
    // state: F64 -> phi[cur] = phi^n, phi[1-cur] = phi^{n-1};
    //        F32K -> phi[cur] (the float part) + lo[cur] (its compensation, 16-bit codes) = phi^n,
    //                dlt[dcur] = phi^n - phi^{n-1}
    //        (dlt[1] exists once temporal blocking is enabled: fused sub-steps read neighbours' dlt, so it ping-pongs)
    void* phi[2];
    void* lo[2];
    void* dlt[2];
    int dcur;
    void* rho;  // stored source s = (c dt)^2 4 pi G (rho - rho_bar), rho_bar = mean(rho) for periodic boundaries, else 0
    int cur;
    double* robin;  // 3 doubles per face ghost: a = nu/mu, r_g, r_i (see boundary.cu)
    float2* robin32;  // alpha, beta rounded to float (compensated float grids)
    double* red;    // reduction scratch
    long long red_elems;
    double* dres;   // small device result buffer
    double* dsum;   // sum(rho) of the last density, written on the device by the source preparation
    int* derr;      // device error word: value 1 a bounded wait in a kernel gave up (HG_ERR_TIMEOUT), value 2 a debug
                    // index check failed (HG_ERR_BOUNDS)
    int mass_pending;  // mass / rho_bar below not yet read back from dsum
    double* staging;  // dense nz*ny*nx doubles, allocated on first host transfer
    double Q[hg::kMaxQ];
    int have_Q;
    double mass, rho_bar;
    long long step;
    int tdepth;
    int texact;  // fused sub-steps bit-identical to single sweeps (hg_set_temporal_exact)
    int ziface;  // bit 0 / bit 1: -z / +z face is an interface to a neighbouring slab (hg_set_z_interface)
    int zb;  // z planes per block of the single sweep (0 = default rule; set by the batch autotuner)
    hg::YlmNorm ylm;
    // measurement: kernel launch count and CUDA events around the sub-step kernel
    long long launches;
    int prof;
    int prof_used;          // event pairs recorded since the last fold
    double prof_ms;         // folded time
    long long prof_count;   // folded launches
    cudaEvent_t* prof_ev;   // 2 * kProfPairs events, created when profiling is first enabled
    // adjoint: a shadow grid (same geometry, precision, boundary condition; zero boundary data and source) that
    // carries lambda, and the running sum of lambda over the reverse sub-steps (float pair or double, padded layout)
    hg_grid* adj;
    void* acc[2];
    // host I/O pipeline (hg_io_step): an upload and a download stream, two slots of device buffers with, per slot,
    // events for "density uploaded", "density consumed", "acceleration written", and a ring of completion events
    // (one per call: its download has finished)
    cudaStream_t io_up, io_down;
    void* io_rho[2];
    void* io_acc[2];
    size_t io_rho_bytes, io_acc_bytes;
    cudaEvent_t io_ev[2][3];
    cudaEvent_t io_done[8];
    long long io_issued, io_waited;
    // TMA tensor maps of the compensated-float state: hi[0..1], lo[0..1], dlt[0..1], s (stencil_tma.cu)
    CUtensorMap tm[7];
    int tm_ready;  // 0: not built, 1: built without dlt[1], 2: built with dlt[1]
    CUtensorMap tm2[7];  // the same arrays with the boxes of the depth-2 kernel (temporal_tma.cu)
    int tm2_ready;
};

namespace hg {

// error reporting (thread-local message)
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define HG_CUDA(call)                                     \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return hg::cuda_fail(e_, #call); \
    } while (0)
// after every kernel launch of a grid `g` in scope: count it and report a launch failure
#define HG_LAUNCHED(what)                                 \
    do {                                                  \
        ++g->launches;                                    \
        cudaError_t e_ = cudaGetLastError();              \
        if (e_ != cudaSuccess) return hg::cuda_fail(e_, what); \
    } while (0)

// kernels' host launchers (each returns HG_OK or an error code)
int launch_step_single(hg_grid* g);                  // one interior sweep: cur -> 1-cur (stencil.cu)
int adjoint_inject(hg_grid* a, const void* v, int vdt);
int adjoint_accumulate(hg_grid* a, void* acc_a, void* acc_b);
int adjoint_gradient(hg_grid* a, const void* acc_a, const void* acc_b, void* out, int odt, double* scratch);
int launch_periodic_fill(hg_grid* g, int b);         // periodic ghosts of time-level buffer b
int launch_temporal(hg_grid* g, int k);              // k fused sub-steps: cur -> 1-cur (temporal.cu)
struct SweepArgs;
int launch_sweep_f32k_tma(hg_grid* g, const SweepArgs& A);  // TMA-staged compensated-float sweep (stencil_tma.cu)
int launch_temporal2_tma(hg_grid* g);                // two fused TMA-staged sub-steps (temporal_tma.cu)
int device_error(hg_grid* g);                        // HG_ERR_TIMEOUT if a kernel's bounded wait gave up (syncs)
// raise a kernel's dynamic shared-memory limit once per device (the attribute is per device); `done` holds one bit
// per device id
int smem_attr_once(const void* fn, int bytes, unsigned long long* done);
int bounds_selftest(hg_grid* g);                     // the debug index check on an index past the array (stencil_tma.cu)
int wait_selftest(hg_grid* g);                       // a wait that cannot complete, then device_error (stencil_tma.cu)
int ensure_staging(hg_grid* g);
int prepare_source(hg_grid* g, const void* src, int dtype);  // dense rho -> stored s, sum(rho) -> dsum (no sync)
int sync_mass(hg_grid* g);                           // dsum -> host mass / rho_bar (syncs once per density)
int set_ghosts_dirichlet(hg_grid* g);                // multipole data into both buffers
int compute_moments(hg_grid* g, const void* rho_dense, int dtype);
int seed_ghosts(hg_grid* g);                         // after hg_set_phi
int reduce_sum(hg_grid* g, const void* dense, int dtype, double* out_dev);
int stats(hg_grid* g, hg_stats* s);
int compare(hg_grid* g, const double* phiP_dense, double out[3]);
int accel(hg_grid* g, void* ax, void* ay, void* az, int dtype);
int unpack_phi(hg_grid* g, void* dst_dense, int dtype);
int unpack_phi_ghosted(hg_grid* g, double* dst);
int set_phi_device(hg_grid* g, const void* phi_dense, const void* prev_dense, int dtype);
constexpr int kProfPairs = 4096;
int prof_begin(hg_grid* g);  // record the start event of a sub-step kernel launch (no-op unless profiling)
int prof_end(hg_grid* g);
int prof_fold(hg_grid* g);   // synchronise and add the recorded pairs to prof_ms

// ---- sweep arguments (stencil.cu) ----
struct Bnd {
    int faces;              // 1: Robin ghosts to update (block epilogue)
    int periodic;           // 1: copy the new boundary cells into the opposite ghosts (block epilogue)
    int xfaces;             // 0, or HG_BC_PERIODIC: the x-face ghost copies are made inside the sweep loop
    int zskip;              // bit 0 / bit 1: the -z / +z face is an interface to a neighbouring slab (its ghost
                            // plane is supplied by the caller before each sub-step and never written by a sweep)
    const float2* robin32;  // (alpha, beta) per face ghost, compensated float grids
    const double* robin;    // (a = nu/mu, r_g, r_i) per face ghost, FP64 grids
    long long off[7];       // face offsets in the ghost enumeration (hg::Faces)
    int* err;               // the grid's device error word (debug index checks)
};

// Everything one sweep of one grid needs (a launch of one grid, or one entry of a batched launch).
struct SweepArgs {
    const void* hi_c;  // phi^n: F64 values, or the float part (F32K)
    const void* lo_c;  // F32K compensation of phi^n
    void* hi_n;        // level n+1 (F64: written over phi^{n-1})
    void* lo_n;
    void* dlt;         // F32K phi^n - phi^{n-1}, updated in place
    const void* rho;   // scaled source s
    Layout L;
    double nu2;
    float nu2f;        // nu^2 rounded to float once (compensated float sweeps)
    int zb;            // z planes per block
    int prec;
    int exact;         // fused sub-steps: inner levels round their compensation as a store and a load would
    int cpl;           // FP64 sweep: x cells per lane (4: 128-cell tile rows; 1: 32-cell rows, for nx that 128 fits badly)
    unsigned gx, gy;   // blocks in x and y of this grid's sweep
    Bnd B;
};

SweepArgs sweep_args(const hg_grid* g, int zb, int cpl = 0);  // sub-step cur -> 1 - cur of grid g; zb = 0: default z
                                                              // chunk; cpl = 0: FP64 cells per lane by tile fit
int f64_cells_per_lane(int nx);  // 4, or 1 when 32-cell tile rows waste fewer lanes than 128-cell ones
// a 3-D TMA map over a padded array (pitch x (ny+2) x (nz+2) elements of `bytes` each), boxes box_x x box_y x 1
int tma_encode(CUtensorMap* m, void* base, const Layout& L, int bytes, int box_x, int box_y);

// One grid of a batched launch: its sweep arguments and, for a compensated-float grid, the tensor maps of its state
// (hi, lo codes, dlt, s of level n) and its error word.
struct alignas(128) TmaEntry {
    CUtensorMap m[4];
    SweepArgs A;
    int* err;
};
int tma_entry(hg_grid* g, TmaEntry* e, int zb = 0);  // compensated-float g's sub-step cur -> 1 - cur (all ghosts in the launch)
int launch_step_batch(cudaStream_t st, const TmaEntry* tab, const unsigned* first, int n, unsigned total_blocks);
// one precision class of a batched sub-step (FP64 entries, or compensated-float entries) as a launch of its own
int launch_batch_class(cudaStream_t st, bool f64, const TmaEntry* tab, const unsigned* first, int n,
                       unsigned total_blocks);
unsigned sweep_blocks(const SweepArgs& A);

// ---- deterministic reductions --------------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // 2 per SM; fixed so that the reduction order, hence the result, is reproducible

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// block sum (or max) of one value per thread; blockDim.x a multiple of 32; result valid in thread 0
__device__ __forceinline__ double block_reduce(double v, double* sh, bool is_max) {
    v = is_max ? warp_max(v) : warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        r = is_max ? warp_max(r) : warp_sum(r);
    }
    return r;
}
__device__ __forceinline__ double block_sum(double v, double* sh) { return block_reduce(v, sh, false); }

long long reduction_scratch_elems();

inline int grid_blocks(long long n, int threads, int cap) {
    long long b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace hg
