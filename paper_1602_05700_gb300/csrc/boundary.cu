// Outer boundary of the hyperbolic gravity solver (arXiv 1602.05700, Sec. 2 and Sec. 4) and the FP64 multipole
// moments of the density.  Only the six face ghost layers are used: the 7-point stencil and the central
// gradient never read edge or corner ghosts.
//
//   Dirichlet (multipole)   phi_g = -G sum_{l<=lmax} 4 pi/(2l+1) sum_m Q_lm r_g^l Y_lm(x_g) / r_g^{2l+1},
//                           Q_lm = sum_cells rho h^3 r^l Y_lm(x), about the coordinate origin; lmax = 0 is the
//                           monopole -G M / r (the analytic mode).  Written once per hg_set_density into both
//                           time levels (rho, hence the data, is frozen during the sub-steps, Sec. 2).
//   Robin                   monopole radiation condition d_t(r phi) + c_h d_r(r phi) = 0, d_r = d_n / mu,
//                           mu = |x_g . n| / r_g, upwinded from the interior neighbour i:
//                           u_g^{n+1} = u_g^n - (nu/mu)(u_g^n - u_i^n), u = r phi (FP64), or equivalently
//                           phi_g^{n+1} = alpha phi_g^n + beta phi_i^n, alpha = 1 - nu/mu, beta = (nu/mu) r_i / r_g
//                           (compensated float).  Its static limit r_g phi_g = r_i phi_i seeds a new state.  The
//                           per-sub-step update is fused into the sweep kernels (stencil.cu, temporal.cu).
//   Periodic                ghost = interior cell on the opposite face; the sweep kernels write these copies (in their
//                           epilogue), the kernel here fills them for a freshly seeded state or an adjoint injection.
//
// r^l Y_lm is evaluated as a polynomial (no trigonometry): with C_m + i S_m = (x + i y)^m,
//   r^l Y_lm = n_lm q_l^m(z, r^2) {C_m (m > 0), 1 (m = 0), S_|m| (m < 0)},
//   q_m^m = (-1)^m (2m-1)!!,  q_{m+1}^m = (2m+1) z q_m^m,
//   q_l^m = ((2l-1) z q_{l-1}^m - (l+m-1) r^2 q_{l-2}^m) / (l - m),
// n_l0 = K_l0, n_lm = sqrt(2) K_lm, K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)  (real orthonormal harmonics with the
// Condon-Shortley phase).
#include <math.h>

#include <mutex>

#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

namespace {

template <int LMAX>
__device__ __forceinline__ void solid_harmonics(double x, double y, double z, const YlmNorm& N,
                                                double R[(LMAX + 1) * (LMAX + 1)]) {
    double C[LMAX + 1], S[LMAX + 1];
    C[0] = 1.0;
    S[0] = 0.0;
#pragma unroll
    for (int m = 1; m <= LMAX; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
    const double r2 = x * x + y * y + z * z;
    double dfact = 1.0;  // (-1)^m (2m-1)!!
#pragma unroll
    for (int m = 0; m <= LMAX; ++m) {
        if (m > 0) dfact *= -(2.0 * m - 1.0);
        double q2 = 0.0, q1 = dfact;  // q_{l-2}^m, q_{l-1}^m
#pragma unroll
        for (int l = m; l <= LMAX; ++l) {
            double q;
            if (l == m) {
                q = dfact;
            } else if (l == m + 1) {
                q = (2.0 * m + 1.0) * z * dfact;
            } else {
                q = ((2.0 * l - 1.0) * z * q1 - (double)(l + m - 1) * r2 * q2) * N.inv_lm[l * l + l + m];
            }
            if (l > m) {
                q2 = q1;
                q1 = q;
            }
            const int base = l * l + l;
            if (m == 0) {
                R[base] = N.n[base] * q;
            } else {
                R[base + m] = N.n[base + m] * q * C[m];
                R[base - m] = N.n[base + m] * q * S[m];
            }
        }
    }
}

__device__ __forceinline__ double load_as_double(const void* p, int dtype, long long i) {
    return dtype == HG_DT_F64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}


// ---- double-double sums of the moments -----------------------------------------------------------------------
// Each moment is a sum over every cell (1.7e7 terms at 256^3).  A plain running or tree sum in FP64 carries a
// rounding error that the lossless scheme then carries, through the Dirichlet data, into phi; so every partial sum
// is kept as an unevaluated pair s + e (TwoSum: s is the rounded sum, e collects the exact rounding errors), whose
// error is of order n eps^2 of the sum of |terms|.  The final s + e, rounded once, is then the correctly rounded
// sum of the terms except in the rare case that the exact sum lies within that tiny error of a midpoint between
// two doubles.
__device__ __forceinline__ void dd_add(double& s, double& e, double x) {
    const double t = __dadd_rn(s, x);
    const double v = __dsub_rn(t, s);
    e = __dadd_rn(e, __dadd_rn(__dsub_rn(s, __dsub_rn(t, v)), __dsub_rn(x, v)));
    s = t;
}
// (s, e) += (s2, e2), renormalised so that s is the rounded value of the pair
__device__ __forceinline__ void dd_merge(double& s, double& e, double s2, double e2) {
    dd_add(s, e, s2);
    e = __dadd_rn(e, e2);
    const double t = __dadd_rn(s, e);
    e = __dsub_rn(e, __dsub_rn(t, s));
    s = t;
}
__device__ __forceinline__ void dd_warp(double& s, double& e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
        dd_merge(s, e, s2, e2);
    }
}
// block sum of one pair per thread (blockDim.x a multiple of 32, at most 1024); result valid in thread 0
__device__ __forceinline__ void dd_block(double& s, double& e, double* sh) {
    dd_warp(s, e);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sh[2 * w] = s;
        sh[2 * w + 1] = e;
    }
    __syncthreads();
    if (w == 0) {
        const bool have = l < (int)(blockDim.x >> 5);
        s = have ? sh[2 * l] : 0.0;
        e = have ? sh[2 * l + 1] : 0.0;
        dd_warp(s, e);
    }
}

constexpr int kMomBlocks = 152;  // fixed, so that the result does not depend on the device

template <int LMAX>
__global__ void __launch_bounds__(kRedThreads) k_moments(const void* rho, int dtype, int nx, int ny, int nz, double h,
                                                         double ox, double oy, double oz, YlmNorm N,
                                                         double* partial) {
    constexpr int NQ = (LMAX + 1) * (LMAX + 1);
    __shared__ double sh[64];
    double as[NQ], ae[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) as[q] = ae[q] = 0.0;
    const long long n = (long long)nx * ny * nz;
    const double h3 = __dmul_rn(__dmul_rn(h, h), h);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const long long r = c / nx;
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const double m = __dmul_rn(load_as_double(rho, dtype, c), h3);
        if (m == 0.0) continue;
        double R[NQ];
        solid_harmonics<LMAX>(ox + (i + 0.5) * h, oy + (j + 0.5) * h, oz + (k + 0.5) * h, N, R);
#pragma unroll
        for (int q = 0; q < NQ; ++q) dd_add(as[q], ae[q], __dmul_rn(m, R[q]));
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double s = as[q], e = ae[q];
        dd_block(s, e, sh);
        if (threadIdx.x == 0) {
            partial[2 * ((long long)blockIdx.x * NQ + q)] = s;
            partial[2 * ((long long)blockIdx.x * NQ + q) + 1] = e;
        }
    }
}

// sum the pairs partial[2 (b nq + q) + {0, 1}] over b in a fixed order (one block); out[q] = the rounded pair
__global__ void __launch_bounds__(kRedThreads) k_finish(const double* partial, int nblocks, int nq, double* out) {
    __shared__ double sh[64];
    for (int q = 0; q < nq; ++q) {
        double s = 0.0, e = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
            dd_merge(s, e, partial[2 * ((long long)b * nq + q)], partial[2 * ((long long)b * nq + q) + 1]);
        dd_block(s, e, sh);
        if (threadIdx.x == 0) out[q] = s;
    }
}

template <int LMAX>
__device__ double multipole_phi(double x, double y, double z, const double* Q, const YlmNorm& N, double G) {
    constexpr int NQ = (LMAX + 1) * (LMAX + 1);
    double R[NQ];
    solid_harmonics<LMAX>(x, y, z, N, R);
    const double r2 = x * x + y * y + z * z;
    const double ir = 1.0 / sqrt(r2);
    const double ir2 = ir * ir;
    double irp = ir;  // r^{-(2l+1)}
    double phi = 0.0;
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
        double s = 0.0;
#pragma unroll
        for (int m = -l; m <= l; ++m) s = fma(Q[l * l + l + m], R[l * l + l + m], s);
        phi = fma(4.0 * 3.14159265358979323846 / (2.0 * l + 1.0) * irp, s, phi);
        irp *= ir2;
    }
    return -G * phi;
}

struct QArr {
    double q[kMaxQ];
};

// write value v (double) into the face ghost q of both time levels
__device__ __forceinline__ void put_ghost(int prec, void* p0, void* p1, void* l0, void* l1, long long q, double v) {
    if (prec == HG_PREC_F64) {
        ((double*)p0)[q] = v;
        ((double*)p1)[q] = v;
    } else {
        float hi;
        lo_t lo;
        split_f32(v, hi, lo);
        ((float*)p0)[q] = hi;
        ((float*)p1)[q] = hi;
        ((lo_t*)l0)[q] = lo;
        ((lo_t*)l1)[q] = lo;
    }
}

template <int LMAX>
__global__ void k_dirichlet(int prec, void* p0, void* p1, void* l0, void* l1, Layout L, Faces F, double h, double ox,
                            double oy, double oz, double G, QArr Q, YlmNorm N) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= F.off[6]) return;
    int gc[3], ic[3];
    face_cell(F, L.nx, L.ny, L.nz, t, gc, ic);
    double v = multipole_phi<LMAX>(ox + (gc[0] + 0.5) * h, oy + (gc[1] + 0.5) * h, oz + (gc[2] + 0.5) * h, Q.q, N, G);
    put_ghost(prec, p0, p1, l0, l1, L.at(gc[0], gc[1], gc[2]), v);
}

__device__ __forceinline__ double read_phi(int prec, const void* p, const void* lo, long long q) {
    if (prec == HG_PREC_F64) return ((const double*)p)[q];
    return join_f32(((const float*)p)[q], ((const lo_t*)lo)[q]);
}
__device__ __forceinline__ void write_phi(int prec, void* p, void* lo, long long q, double v) {
    if (prec == HG_PREC_F64) {
        ((double*)p)[q] = v;
    } else {
        float hi;
        lo_t l;
        split_f32(v, hi, l);
        ((float*)p)[q] = hi;
        ((lo_t*)lo)[q] = l;
    }
}

// Robin static limit r_g phi_g = r_i phi_i on one time level: phi_g = (phi_i r_i) / r_g
__global__ void k_robin_static(int prec, void* p, void* lo, Layout L, Faces F, const double* __restrict__ coef) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= F.off[6]) return;
    int gc[3], ic[3];
    face_cell(F, L.nx, L.ny, L.nz, t, gc, ic);
    const long long qg = L.at(gc[0], gc[1], gc[2]), qi = L.at(ic[0], ic[1], ic[2]);
    write_phi(prec, p, lo, qg, __ddiv_rn(__dmul_rn(read_phi(prec, p, lo, qi), coef[3 * t + 2]), coef[3 * t + 1]));
}

// periodic copy into the face ghosts of one time level
__device__ __forceinline__ void periodic_ghost(int prec, void* p, void* lo, const Layout& L, const Faces& F, long long t) {
    int gc[3], ic[3];
    int f = face_cell(F, L.nx, L.ny, L.nz, t, gc, ic);
    int src[3] = {gc[0], gc[1], gc[2]};
    int n[3] = {L.nx, L.ny, L.nz};
    src[f / 2] = (f % 2) ? 0 : n[f / 2] - 1;
    const long long qg = L.at(gc[0], gc[1], gc[2]), qs = L.at(src[0], src[1], src[2]);
    if (prec == HG_PREC_F64) {
        ((double*)p)[qg] = ((const double*)p)[qs];
    } else {
        ((float*)p)[qg] = ((const float*)p)[qs];
        ((lo_t*)lo)[qg] = ((const lo_t*)lo)[qs];
    }
}

__global__ void k_periodic(int prec, void* p, void* lo, Layout L, Faces F) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= F.off[6]) return;
    periodic_ghost(prec, p, lo, L, F, t);
}

template <int LMAX>
int run_moments(hg_grid* g, const void* rho, int dtype) {
    constexpr int NQ = (LMAX + 1) * (LMAX + 1);
    k_moments<LMAX><<<kMomBlocks, kRedThreads, 0, g->stream>>>(rho, dtype, g->nx, g->ny, g->nz, g->h, g->origin[0],
                                                                g->origin[1], g->origin[2], g->ylm, g->red);
    HG_LAUNCHED("multipole moment kernel");
    k_finish<<<1, kRedThreads, 0, g->stream>>>(g->red, kMomBlocks, NQ, g->dres);
    HG_LAUNCHED("moment finish kernel");
    return HG_OK;
}

template <int LMAX>
int run_dirichlet(hg_grid* g) {
    QArr Q;
    for (int q = 0; q < kMaxQ; ++q) Q.q[q] = q < (LMAX + 1) * (LMAX + 1) ? g->Q[q] : 0.0;
    long long n = g->F.off[6];
    int threads = 128;
    k_dirichlet<LMAX><<<(unsigned)((n + threads - 1) / threads), threads, 0, g->stream>>>(
        g->prec, g->phi[0], g->phi[1], g->lo[0], g->lo[1], g->L, g->F, g->h, g->origin[0], g->origin[1],
        g->origin[2], g->G, Q, g->ylm);
    HG_LAUNCHED("Dirichlet ghost kernel");
    return HG_OK;
}

}  // namespace

long long reduction_scratch_elems() {
    const long long a = (long long)kRedBlocks * kMaxQ, b = 2LL * kMomBlocks * kMaxQ;
    return a > b ? a : b;
}

int compute_moments(hg_grid* g, const void* rho_dense, int dtype) {
    int rc;
    switch (g->lmax) {
        case 0: rc = run_moments<0>(g, rho_dense, dtype); break;
        case 1: rc = run_moments<1>(g, rho_dense, dtype); break;
        case 2: rc = run_moments<2>(g, rho_dense, dtype); break;
        case 3: rc = run_moments<3>(g, rho_dense, dtype); break;
        case 4: rc = run_moments<4>(g, rho_dense, dtype); break;
        case 5: rc = run_moments<5>(g, rho_dense, dtype); break;
        case 6: rc = run_moments<6>(g, rho_dense, dtype); break;
        case 7: rc = run_moments<7>(g, rho_dense, dtype); break;
        default: rc = run_moments<8>(g, rho_dense, dtype); break;
    }
    if (rc != HG_OK) return rc;
    int nq = (g->lmax + 1) * (g->lmax + 1);
    HG_CUDA(cudaMemcpyAsync(g->Q, g->dres, nq * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    for (int q = nq; q < kMaxQ; ++q) g->Q[q] = 0.0;
    g->have_Q = 1;
    return HG_OK;
}

int set_ghosts_dirichlet(hg_grid* g) {
    switch (g->lmax) {
        case 0: return run_dirichlet<0>(g);
        case 1: return run_dirichlet<1>(g);
        case 2: return run_dirichlet<2>(g);
        case 3: return run_dirichlet<3>(g);
        case 4: return run_dirichlet<4>(g);
        case 5: return run_dirichlet<5>(g);
        case 6: return run_dirichlet<6>(g);
        case 7: return run_dirichlet<7>(g);
        default: return run_dirichlet<8>(g);
    }
}

// periodic copies into the face ghosts of time-level buffer b
int launch_periodic_fill(hg_grid* g, int b) {
    long long n = g->F.off[6];
    int threads = 256;
    unsigned blocks = (unsigned)((n + threads - 1) / threads);
    k_periodic<<<blocks, threads, 0, g->stream>>>(g->prec, g->phi[b], g->lo[b], g->L, g->F);
    HG_LAUNCHED("periodic ghost kernel");
    return HG_OK;
}

// ghosts of a freshly seeded state (both time levels)
int seed_ghosts(hg_grid* g) {
    long long n = g->F.off[6];
    int threads = 256;
    unsigned blocks = (unsigned)((n + threads - 1) / threads);
    for (int b = 0; b < 2; ++b) {
        if (g->bc == HG_BC_ROBIN) {
            k_robin_static<<<blocks, threads, 0, g->stream>>>(g->prec, g->phi[b], g->lo[b], g->L, g->F, g->robin);
            HG_LAUNCHED("Robin static ghost kernel");
        } else if (g->bc == HG_BC_PERIODIC) {
            k_periodic<<<blocks, threads, 0, g->stream>>>(g->prec, g->phi[b], g->lo[b], g->L, g->F);
            HG_LAUNCHED("periodic ghost kernel");
        }
    }
    if (g->bc == HG_BC_DIRICHLET_ANALYTIC || g->bc == HG_BC_DIRICHLET_MULTIPOLE) {
        if (g->have_Q) return set_ghosts_dirichlet(g);
    }
    return HG_OK;
}

}  // namespace hg

// ---- multipole moments without device allocation -------------------------------------------------------------
// The paper has no counterpart to this: it is an entry point for callers that may not allocate GPU memory (see
// hg_moments_noalloc in hg.h).  It runs the same moment and finishing kernels as hg_set_density, with the per-block
// partial sums in a scratch array compiled into the library instead of in memory owned by a grid.
namespace hg {
namespace {

// partial sums (pairs) of kMomBlocks blocks for up to kMaxQ moments, then kMaxQ doubles for a result bound for host
// memory: (2 * 152 * 81 + 81) doubles = 197,640 bytes on every GPU that loads the library, held until the process
// exits
constexpr int kNoAllocDoubles = 2 * kMomBlocks * kMaxQ + kMaxQ;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocDevices];            // device address of the scratch, per device, found on first use
unsigned long long g_noalloc_ctx[kNoAllocDevices];  // id of the CUDA context the address belongs to

// id of the current CUDA context (0 if it cannot be read).  A cudaDeviceReset ends the device's primary context and
// the next runtime call creates a new one, in which the library's module -- and so the array -- may be placed at
// another address; a changed id makes the lookup below run again instead of handing a stale address to a kernel.
unsigned long long current_context_id() {
    typedef int (*get_ctx_t)(void**);
    typedef int (*get_id_t)(void*, unsigned long long*);
    static get_ctx_t get_ctx = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = (get_ctx_t)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)p;
        looked_up = true;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_ctx || !get_id || get_ctx(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// The host name of g_noalloc_scratch is only a stand-in: the kernels need the device address, looked up with the
// device current (the runtime makes its context current first) and cached per device and context.
int noalloc_scratch(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocDevices) return fail(HG_ERR_ARG, "device index %d out of range", dev);
    const unsigned long long ctx = current_context_id();  // 0 while no context is current yet
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev] || ctx != g_noalloc_ctx[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);  // also creates the context on a first call
        if (e != cudaSuccess) {
            g_noalloc_addr[dev] = nullptr;
            return cuda_fail(e, "cudaGetSymbolAddress(moment scratch)");
        }
        g_noalloc_addr[dev] = p;
        g_noalloc_ctx[dev] = current_context_id();
    }
    *out = g_noalloc_addr[dev];
    return HG_OK;
}

template <int LMAX>
int noalloc_moments(const void* rho, int dtype, int nx, int ny, int nz, double h, const double* o, double* scratch,
                    double* Qdev, cudaStream_t st) {
    constexpr int NQ = (LMAX + 1) * (LMAX + 1);
    YlmNorm N;
    fill_ylm_norms(N);
    k_moments<LMAX><<<kMomBlocks, kRedThreads, 0, st>>>(rho, dtype, nx, ny, nz, h, o[0], o[1], o[2], N, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "multipole moment kernel");
    k_finish<<<1, kRedThreads, 0, st>>>(scratch, kMomBlocks, NQ, Qdev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "moment finish kernel");
    return HG_OK;
}

}  // namespace
}  // namespace hg

extern "C" int hg_moments_noalloc(const void* rho, int dtype, int nx, int ny, int nz, double h, const double origin[3],
                                  int lmax, double* Q, int Q_on_device, void* cuda_stream) {
    HG_RANGE("hg_moments_noalloc");
    using namespace hg;
    if (!rho || !Q || !origin) return fail(HG_ERR_ARG, "null pointer");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    if (nx < 1 || ny < 1 || nz < 1) return fail(HG_ERR_ARG, "grid sizes must be >= 1 (got %d %d %d)", nx, ny, nz);
    if (!(h > 0.0) || !isfinite(h) || !isfinite(origin[0]) || !isfinite(origin[1]) || !isfinite(origin[2]))
        return fail(HG_ERR_ARG, "h must be positive and finite, origin finite");
    if (lmax < 0 || lmax > HG_MAX_LMAX)
        return fail(HG_ERR_ARG, "lmax = %d exceeds the fixed scratch of hg_moments_noalloc (sized for lmax <= %d)", lmax,
                    HG_MAX_LMAX);
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* Qdev = Q_on_device ? Q : scratch + 2LL * kMomBlocks * kMaxQ;
    switch (lmax) {
        case 0: rc = noalloc_moments<0>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 1: rc = noalloc_moments<1>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 2: rc = noalloc_moments<2>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 3: rc = noalloc_moments<3>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 4: rc = noalloc_moments<4>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 5: rc = noalloc_moments<5>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 6: rc = noalloc_moments<6>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        case 7: rc = noalloc_moments<7>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
        default: rc = noalloc_moments<8>(rho, dtype, nx, ny, nz, h, origin, scratch, Qdev, st); break;
    }
    if (rc) return rc;
    if (!Q_on_device) {
        const size_t bytes = (size_t)(lmax + 1) * (lmax + 1) * sizeof(double);
        cudaError_t e = cudaMemcpyAsync(Q, Qdev, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "copy of the moments to host memory");
    }
    return HG_OK;
}

