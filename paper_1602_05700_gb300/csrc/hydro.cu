// Ideal-gas hydrodynamics that consumes the hyperbolic self-gravity (arXiv 1602.05700, Sec. 2): the C ABI of
// include/hg_hydro.h, the FP64 stage kernel, the set-up conversion and the FP64 reductions (characteristic speed,
// the virial sums of the paper's Eq. VC).  The stage kernel itself is in hydro_kernels.cuh.
//
// This file is compiled without floating-point contraction (-fmad=false, set by the builder): the FP64 instance
// then rounds every operation exactly as written, and the operation order is the one the ABI header fixes, so
// double-precision states reproduce a plain sequential evaluation of the same formulas bit for bit.  The FP32
// stage kernel is instantiated in hydro_f32.cu with contraction on.
#include <cuda_runtime.h>
#include <math.h>

#include "hg_hydro.h"
#include "hg_internal.cuh"
#include "hydro_kernels.cuh"

struct hg_hydro {
    int nx, ny, nz;
    long long n;  // cells
    double h, gamma, rho_floor, p_floor;
    int dtype, esize;
    cudaStream_t stream;
    int device;
    void* U;         // conserved state, 5 planes
    void* U1;        // stage-1 state, 5 planes
    void* A;         // acceleration, 3 planes (also the double potential for the virial sums)
    void* staging;   // host transfers (5 planes of the larger element type), allocated on first use
    double* red;     // reduction partials
    double* dres;    // reduction results
    long long launches;
    // stage-kernel timing (hg_hydro_profile): event pairs around each stage launch, folded into prof_ms when read
    int prof, prof_used;
    double prof_ms;
    long long prof_count;
    cudaEvent_t* prof_ev;
};

namespace {

using hg::fail;

constexpr int kVirialSums = 5;  // sum rho phi, sum e_int, sum e_kin, sum rho (bound cells), max rho

template <typename Tin, typename T>
__global__ void k_prim_to_cons(const Tin* __restrict__ W, T* __restrict__ U, long long n, T gm1) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T w[5], u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) w[q] = (T)W[q * n + c];
        prim_to_cons(gm1, w, u);
#pragma unroll
        for (int q = 0; q < 5; ++q) U[q * n + c] = u[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(hg::kRedThreads) k_max_speed(const T* __restrict__ U, long long n, T gamma, T gm1,
                                                              double* __restrict__ red) {
    __shared__ double sh[32];
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T u[5], w[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = U[q * n + c];
        cons_to_prim(gm1, u, w);
        const T s = sqrt((w[1] * w[1] + w[2] * w[2]) + w[3] * w[3]) + sqrt(gamma * w[4] / w[0]);
        if ((double)s > m) m = (double)s;
    }
    m = hg::block_reduce(m, sh, true);
    if (threadIdx.x == 0) red[blockIdx.x] = m;
}

// per-block partial sums over the bound cells (E + rho phi < 0), accumulated in FP64.  The kinetic energy of a cell
// is |m|^2 / (2 rho), one division (FP64 division is a long instruction sequence on this GPU), in the state's
// precision: the sums are compared with a sequential FP64 evaluation within a relative tolerance, not bit for bit.
template <typename T>
__global__ void __launch_bounds__(hg::kRedThreads) k_virial(const T* __restrict__ U, const double* __restrict__ phi,
                                                           long long n, double* __restrict__ red) {
    __shared__ double sh[32];
    double acc[kVirialSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const T r = U[c], m1 = U[n + c], m2 = U[2 * n + c], m3 = U[3 * n + c], E = U[4 * n + c];
        const double rd = (double)r;
        if (rd > acc[4]) acc[4] = rd;
        const double rp = rd * phi[c];
        if ((double)E + rp < 0.0) {
            const double ke = (double)(T(0.5) * hdiv((m1 * m1 + m2 * m2) + m3 * m3, r));
            acc[0] += rp;
            acc[1] += (double)E - ke;
            acc[2] += ke;
            acc[3] += rd;
        }
    }
#pragma unroll
    for (int s = 0; s < kVirialSums; ++s) {
        const double v = hg::block_reduce(acc[s], sh, s == 4);
        if (threadIdx.x == 0) red[s * hg::kRedBlocks + blockIdx.x] = v;
        __syncthreads();
    }
}

// fixed-order combination of the per-block partials: nsum arrays, the last `nmax` of them maxima
__global__ void __launch_bounds__(hg::kRedThreads) k_finish(const double* __restrict__ red, int parts, int narr, int nmax,
                                                           double* __restrict__ out) {
    __shared__ double sh[32];
    for (int s = 0; s < narr; ++s) {
        const bool is_max = s >= narr - nmax;
        double v = 0.0;  // every summed or maximised quantity here is >= 0 or a plain sum
        for (int b = threadIdx.x; b < parts; b += blockDim.x) {
            const double x = red[s * parts + b];
            v = is_max ? (x > v ? x : v) : v + x;
        }
        v = hg::block_reduce(v, sh, is_max);
        if (threadIdx.x == 0) out[s] = v;
        __syncthreads();
    }
}

#define HH_LAUNCHED(what)                                       \
    do {                                                        \
        ++H->launches;                                          \
        cudaError_t e_ = cudaGetLastError();                    \
        if (e_ != cudaSuccess) return hg::cuda_fail(e_, what);  \
    } while (0)

int check_hydro(const hg_hydro* H) {
    if (!H) return fail(HG_ERR_ARG, "null hydro state");
    cudaError_t e = cudaSetDevice(H->device);
    if (e != cudaSuccess) return hg::cuda_fail(e, "cudaSetDevice");
    return HG_OK;
}

int ensure_hydro_staging(hg_hydro* H) {
    if (!H->staging) HG_CUDA(cudaMalloc(&H->staging, (size_t)H->n * 5 * sizeof(double)));
    return HG_OK;
}

// z planes per block: about 1200 blocks in total (several waves of the 152 SMs), at least 8 planes per block
int stage_zb(const hg_hydro* H) {
    const long long nxy = (long long)((H->nx + TX - 1) / TX) * ((H->ny + TY - 1) / TY);
    long long zb = (H->nz * nxy + 1199) / 1200;
    if (zb < 8) zb = 8;
    if (zb > H->nz) zb = H->nz;
    return (int)zb;
}

constexpr int kHydroProfPairs = 1024;

int hydro_prof_fold(hg_hydro* H) {
    if (!H->prof_used) return HG_OK;
    HG_CUDA(cudaStreamSynchronize(H->stream));
    for (int p = 0; p < H->prof_used; ++p) {
        float ms = 0.f;
        HG_CUDA(cudaEventElapsedTime(&ms, H->prof_ev[2 * p], H->prof_ev[2 * p + 1]));
        H->prof_ms += ms;
    }
    H->prof_count += H->prof_used;
    H->prof_used = 0;
    return HG_OK;
}

int launch_stage_any(hg_hydro* H, int stage, const void* Uin, const void* U0, const void* A, void* Uout, double dt) {
    hg::HydroStageLaunch L;
    L.stream = H->stream;
    L.nx = H->nx;
    L.ny = H->ny;
    L.nz = H->nz;
    L.zb = stage_zb(H);
    L.stage = stage;
    L.n = H->n;
    L.h = H->h;
    L.gamma = H->gamma;
    L.rho_floor = H->rho_floor;
    L.p_floor = H->p_floor;
    L.dt = dt;
    L.Uin = Uin;
    L.U0 = U0;
    L.A = A;
    L.Uout = Uout;
    if (H->prof) {
        if (H->prof_used == kHydroProfPairs) {
            int rc = hydro_prof_fold(H);
            if (rc) return rc;
        }
        HG_CUDA(cudaEventRecord(H->prof_ev[2 * H->prof_used], H->stream));
    }
    const cudaError_t e = H->dtype == HG_DT_F64 ? hg::hydro_stage_f64(L) : hg::hydro_stage_f32(L);
    ++H->launches;
    if (e != cudaSuccess) return hg::cuda_fail(e, "k_hydro_stage");
    if (H->prof) {
        HG_CUDA(cudaEventRecord(H->prof_ev[2 * H->prof_used + 1], H->stream));
        ++H->prof_used;
    }
    return HG_OK;
}

int prim_to_cons_launch(hg_hydro* H, const void* W, int dtype) {
    const int blocks = hg::grid_blocks(H->n, 256, 152 * 8);
    if (H->dtype == HG_DT_F64) {
        const double gm1 = H->gamma - 1.0;
        if (dtype == HG_DT_F64) k_prim_to_cons<double, double><<<blocks, 256, 0, H->stream>>>((const double*)W, (double*)H->U, H->n, gm1);
        else k_prim_to_cons<float, double><<<blocks, 256, 0, H->stream>>>((const float*)W, (double*)H->U, H->n, gm1);
    } else {
        const float gm1 = (float)(H->gamma - 1.0);
        if (dtype == HG_DT_F64) k_prim_to_cons<double, float><<<blocks, 256, 0, H->stream>>>((const double*)W, (float*)H->U, H->n, gm1);
        else k_prim_to_cons<float, float><<<blocks, 256, 0, H->stream>>>((const float*)W, (float*)H->U, H->n, gm1);
    }
    HH_LAUNCHED("k_prim_to_cons");
    return HG_OK;
}

int check_pair(const hg_hydro* H, const hg_grid* g) {
    if (g->nx != H->nx || g->ny != H->ny || g->nz != H->nz)
        return fail(HG_ERR_ARG, "gravity grid %dx%dx%d does not match the hydro grid %dx%dx%d", g->nx, g->ny, g->nz,
                    H->nx, H->ny, H->nz);
    if (g->stream != H->stream) return fail(HG_ERR_ARG, "the gravity grid and the hydro state use different streams");
    if (g->device != H->device) return fail(HG_ERR_ARG, "the gravity grid and the hydro state are on different devices");
    return HG_OK;
}

void release(hg_hydro* H) {
    void* ptrs[] = {H->U, H->U1, H->A, H->staging, H->red, H->dres};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (H->prof_ev) {
        for (int e = 0; e < 2 * kHydroProfPairs; ++e)
            if (H->prof_ev[e]) cudaEventDestroy(H->prof_ev[e]);
        delete[] H->prof_ev;
    }
}

}  // namespace

namespace hg {
cudaError_t hydro_stage_f64(const HydroStageLaunch& L) { return launch_hydro_stage<double>(L); }
}  // namespace hg

extern "C" {

int hg_hydro_init(hg_hydro** out, int nx, int ny, int nz, double h, double gamma, double rho_floor, double p_floor,
                  int dtype, void* cuda_stream) {
    HG_RANGE("hg_hydro_init");
    if (!out) return fail(HG_ERR_ARG, "null output handle");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(HG_ERR_ARG, "grid sizes must be >= 1 (got %d %d %d)", nx, ny, nz);
    if ((long long)(ny + TY - 1) / TY > 65535) return fail(HG_ERR_ARG, "ny too large");
    if (!(h > 0.0)) return fail(HG_ERR_ARG, "h must be > 0");
    if (!(gamma > 1.0)) return fail(HG_ERR_ARG, "gamma must be > 1");
    if (!(rho_floor >= 0.0) || !(p_floor >= 0.0)) return fail(HG_ERR_ARG, "floors must be >= 0");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    hg_hydro* H = new hg_hydro();
    H->nx = nx;
    H->ny = ny;
    H->nz = nz;
    H->n = (long long)nx * ny * nz;
    H->h = h;
    H->gamma = gamma;
    H->rho_floor = rho_floor;
    H->p_floor = p_floor;
    H->dtype = dtype;
    H->esize = dtype == HG_DT_F64 ? 8 : 4;
    H->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&H->device);
    const size_t fb = (size_t)H->n * H->esize;
    if (e == cudaSuccess) e = cudaMalloc(&H->U, 5 * fb);
    if (e == cudaSuccess) e = cudaMalloc(&H->U1, 5 * fb);
    if (e == cudaSuccess) e = cudaMalloc(&H->A, 3 * fb);
    if (e == cudaSuccess) e = cudaMalloc(&H->red, (size_t)kVirialSums * hg::kRedBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->dres, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(H->U, 0, 5 * fb, H->stream);
    if (e != cudaSuccess) {
        release(H);
        delete H;
        return hg::cuda_fail(e, "hg_hydro_init");
    }
    *out = H;
    return HG_OK;
}

int hg_hydro_set_primitive(hg_hydro* H, const void* W, int dtype, int on_device) {
    HG_RANGE("hg_hydro_set_primitive");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!W) return fail(HG_ERR_ARG, "null primitive fields");
    if (dtype != HG_DT_F32 && dtype != HG_DT_F64) return fail(HG_ERR_ARG, "unknown dtype %d", dtype);
    const void* src = W;
    if (!on_device) {
        if ((rc = ensure_hydro_staging(H))) return rc;
        HG_CUDA(cudaMemcpyAsync(H->staging, W, (size_t)H->n * 5 * (dtype == HG_DT_F64 ? 8 : 4),
                                cudaMemcpyHostToDevice, H->stream));
        src = H->staging;
    }
    if ((rc = prim_to_cons_launch(H, src, dtype))) return rc;
    if (!on_device) HG_CUDA(cudaStreamSynchronize(H->stream));
    return HG_OK;
}

int hg_hydro_set_state(hg_hydro* H, const void* U, int dtype, int on_device) {
    HG_RANGE("hg_hydro_set_state");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!U) return fail(HG_ERR_ARG, "null state");
    if (dtype != H->dtype) return fail(HG_ERR_ARG, "state dtype %d does not match the hydro precision %d", dtype, H->dtype);
    HG_CUDA(cudaMemcpyAsync(H->U, U, (size_t)H->n * 5 * H->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, H->stream));
    if (!on_device) HG_CUDA(cudaStreamSynchronize(H->stream));
    return HG_OK;
}

int hg_hydro_get_state(hg_hydro* H, void* U, int dtype, int on_device) {
    HG_RANGE("hg_hydro_get_state");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!U) return fail(HG_ERR_ARG, "null output");
    if (dtype != H->dtype) return fail(HG_ERR_ARG, "state dtype %d does not match the hydro precision %d", dtype, H->dtype);
    HG_CUDA(cudaMemcpyAsync(U, H->U, (size_t)H->n * 5 * H->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, H->stream));
    if (!on_device) HG_CUDA(cudaStreamSynchronize(H->stream));
    return HG_OK;
}

int hg_hydro_max_speed(hg_hydro* H, double* s) {
    HG_RANGE("hg_hydro_max_speed");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!s) return fail(HG_ERR_ARG, "null output");
    if (H->dtype == HG_DT_F64)
        k_max_speed<double><<<hg::kRedBlocks, hg::kRedThreads, 0, H->stream>>>((const double*)H->U, H->n, H->gamma,
                                                                                H->gamma - 1.0, H->red);
    else
        k_max_speed<float><<<hg::kRedBlocks, hg::kRedThreads, 0, H->stream>>>((const float*)H->U, H->n, (float)H->gamma,
                                                                               (float)(H->gamma - 1.0), H->red);
    HH_LAUNCHED("k_max_speed");
    k_finish<<<1, hg::kRedThreads, 0, H->stream>>>(H->red, hg::kRedBlocks, 1, 1, H->dres);
    HH_LAUNCHED("k_finish");
    HG_CUDA(cudaMemcpyAsync(s, H->dres, sizeof(double), cudaMemcpyDeviceToHost, H->stream));
    HG_CUDA(cudaStreamSynchronize(H->stream));
    return HG_OK;
}

int hg_hydro_step(hg_hydro* H, hg_grid* g, double dt, int n_substeps) {
    HG_RANGE("hg_hydro_step");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!(dt > 0.0)) return fail(HG_ERR_ARG, "dt must be > 0");
    const void* A = nullptr;
    if (g) {
        if (n_substeps < 0) return fail(HG_ERR_ARG, "n_substeps must be >= 0");
        if ((rc = check_pair(H, g))) return rc;
        if ((rc = hg_set_density(g, H->U, H->dtype, 1))) return rc;  // plane 0 of the state is rho
        if ((rc = hg_step(g, n_substeps))) return rc;
        const size_t fb = (size_t)H->n * H->esize;
        if ((rc = hg_accel(g, H->A, (char*)H->A + fb, (char*)H->A + 2 * fb, H->dtype))) return rc;
        A = H->A;
    }
    if ((rc = launch_stage_any(H, 1, H->U, nullptr, A, H->U1, dt))) return rc;
    return launch_stage_any(H, 2, H->U1, H->U, A, H->U, dt);
}

int hg_hydro_virial(hg_hydro* H, hg_grid* g, double out[6]) {
    HG_RANGE("hg_hydro_virial");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (!g || !out) return fail(HG_ERR_ARG, "null grid or output");
    if ((rc = check_pair(H, g))) return rc;
    double* phi = (double*)H->A;  // 3 planes of the state's type hold at least one plane of doubles
    if ((rc = hg::unpack_phi(g, phi, HG_DT_F64))) return rc;
    if (H->dtype == HG_DT_F64)
        k_virial<double><<<hg::kRedBlocks, hg::kRedThreads, 0, H->stream>>>((const double*)H->U, phi, H->n, H->red);
    else
        k_virial<float><<<hg::kRedBlocks, hg::kRedThreads, 0, H->stream>>>((const float*)H->U, phi, H->n, H->red);
    HH_LAUNCHED("k_virial");
    k_finish<<<1, hg::kRedThreads, 0, H->stream>>>(H->red, hg::kRedBlocks, kVirialSums, 1, H->dres);
    HH_LAUNCHED("k_finish");
    double r[kVirialSums];
    HG_CUDA(cudaMemcpyAsync(r, H->dres, sizeof(r), cudaMemcpyDeviceToHost, H->stream));
    HG_CUDA(cudaStreamSynchronize(H->stream));
    const double h3 = H->h * H->h * H->h;
    const double W = 0.5 * r[0] * h3;
    const double Ui = r[1] * h3;
    out[0] = W;
    out[1] = Ui;
    out[2] = r[2] * h3;
    out[3] = (W + 3.0 * (H->gamma - 1.0) * Ui) / fabs(W);
    out[4] = r[4];
    out[5] = r[3] * h3;
    return HG_OK;
}

int hg_hydro_launches(hg_hydro* H, long long* n) {
    HG_RANGE("hg_hydro_launches");
    if (!H || !n) return fail(HG_ERR_ARG, "null argument");
    *n = H->launches;
    return HG_OK;
}

int hg_hydro_profile(hg_hydro* H, int enable) {
    HG_RANGE("hg_hydro_profile");
    int rc = check_hydro(H);
    if (rc) return rc;
    if (enable && !H->prof_ev) {
        H->prof_ev = new cudaEvent_t[2 * kHydroProfPairs]();
        for (int e = 0; e < 2 * kHydroProfPairs; ++e) HG_CUDA(cudaEventCreate(&H->prof_ev[e]));
    }
    if (!enable && (rc = hydro_prof_fold(H))) return rc;
    H->prof = enable ? 1 : 0;
    return HG_OK;
}

int hg_hydro_profile_read(hg_hydro* H, double* stage_ms, long long* stage_launches) {
    HG_RANGE("hg_hydro_profile_read");
    int rc = check_hydro(H);
    if (rc) return rc;
    if ((rc = hydro_prof_fold(H))) return rc;
    if (stage_ms) *stage_ms = H->prof_ms;
    if (stage_launches) *stage_launches = H->prof_count;
    H->prof_ms = 0.0;
    H->prof_count = 0;
    return HG_OK;
}

void hg_hydro_free(hg_hydro* H) {
    HG_RANGE("hg_hydro_free");
    if (!H) return;
    cudaSetDevice(H->device);
    cudaStreamSynchronize(H->stream);
    release(H);
    delete H;
}

}  // extern "C"
