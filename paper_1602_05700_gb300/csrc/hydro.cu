// Ideal-gas hydrodynamics that consumes the hyperbolic self-gravity (arXiv 1602.05700, Sec. 2): finite volume,
// minmod-limited piecewise-linear primitives, HLLC fluxes with Davis' wave-speed bounds, outgoing (zero-gradient)
// boundaries, two-stage SSP Runge-Kutta with the gravity source (0, rho a, m . a), and the virial measure of the
// paper's Eq. VC.  The ABI is include/hg_hydro.h.
//
// This file is compiled without floating-point contraction (-fmad=false, set by the builder): the FP64 instance
// then rounds every operation exactly as written, and the operation order below is the one the ABI header fixes,
// so double-precision states reproduce a plain sequential evaluation of the same formulas bit for bit.
//
// Kernel design (one launch per Runge-Kutta stage): a block owns a 32 x 8 column of cells and marches along z
// through a chunk of planes.  A ring of four primitive planes (the column plus a 2-cell halo in x and y) sits in
// shared memory; each plane of the global state is read once per block and converted to primitives once.  Every
// face flux is evaluated once: the 33 x 8 x-faces and 32 x 9 y-faces of the current plane go to shared memory,
// the z-face above each cell is kept in registers and becomes the next plane's lower face.  The update, the
// gravity source, the stage combination and the floors are fused into the same pass, so a stage reads the stage
// state (and, for stage 2, the step's initial state and a) once and writes the new state once.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <vector>

#include "hg_hydro.h"
#include "hg_internal.cuh"

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
};

namespace {

using hg::fail;

constexpr int TX = 32, TY = 8, NT = TX * TY, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO, PCELLS = PX * PY;  // 36 x 12 cells per staged plane
constexpr int NXF = (TX + 1) * TY;  // x-faces of one plane of the column
constexpr int NYF = TX * (TY + 1);  // y-faces
constexpr int kVirialSums = 5;      // sum rho phi, sum e_int, sum e_kin, sum rho (bound cells), max rho

template <typename T>
struct Smem {
    T w[4][5][PCELLS];  // primitive planes k-1 .. k+2 (ring by plane index mod 4)
    T fx[5][NXF];
    T fy[5][NYF];
};

template <typename T>
struct Gas {
    T gamma, gm1, rho_floor, p_floor;
};

template <typename T>
struct StageArgs {
    const T* __restrict__ Uin;  // stage state
    const T* U0;                // the step's initial state (stage 2; may be Uout: each cell is read, then written,
                                // by the same thread, so neither pointer is restrict nor read through the nc path)
    const T* __restrict__ A;    // acceleration (3 planes) or null
    T* Uout;
    long long n;
    int nx, ny, nz, zb;
    T dt, inv_h;
    Gas<T> gas;
};

__device__ __forceinline__ int slot(int p) { return (p + 4) & 3; }  // p >= -2

template <typename T>
__device__ __forceinline__ T kinetic(const T u[5], T& vx, T& vy, T& vz) {
    vx = u[1] / u[0];
    vy = u[2] / u[0];
    vz = u[3] / u[0];
    return T(0.5) * ((u[1] * vx + u[2] * vy) + u[3] * vz);
}

template <typename T>
__device__ __forceinline__ void cons_to_prim(T gm1, const T u[5], T w[5]) {
    T vx, vy, vz;
    const T ke = kinetic(u, vx, vy, vz);
    w[0] = u[0];
    w[1] = vx;
    w[2] = vy;
    w[3] = vz;
    w[4] = gm1 * (u[4] - ke);
}

template <typename T>
__device__ __forceinline__ void prim_to_cons(T gm1, const T w[5], T u[5]) {
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = w[4] / gm1 + T(0.5) * w[0] * ((w[1] * w[1] + w[2] * w[2]) + w[3] * w[3]);
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

// conserved state u and physical flux f along axis D of the primitive state w
template <typename T, int D>
__device__ __forceinline__ void state_flux(T gm1, const T w[5], T u[5], T f[5]) {
    prim_to_cons(gm1, w, u);
    const T un = w[1 + D];
    const T mf = w[0] * un;
    f[0] = mf;
    f[1] = mf * w[1];
    f[2] = mf * w[2];
    f[3] = mf * w[3];
    f[1 + D] = f[1 + D] + w[4];
    f[4] = (u[4] + w[4]) * un;
}

// HLLC flux along axis D between primitive states wl and wr (Davis bounds, Toro-Spruce-Speares star states)
template <typename T, int D>
__device__ __forceinline__ void hllc(const Gas<T>& G, const T wl[5], const T wr[5], T F[5]) {
    T ul[5], fl[5], ur[5], fr[5];
    state_flux<T, D>(G.gm1, wl, ul, fl);
    state_flux<T, D>(G.gm1, wr, ur, fr);
    const T al = sqrt(G.gamma * wl[4] / wl[0]);
    const T ar = sqrt(G.gamma * wr[4] / wr[0]);
    const T unl = wl[1 + D], unr = wr[1 + D];
    const T a1 = unl - al, a2 = unr - ar, b1 = unl + al, b2 = unr + ar;
    const T sl = a1 < a2 ? a1 : a2;
    const T sr = b1 > b2 ? b1 : b2;
    if (sl >= T(0)) {
#pragma unroll
        for (int q = 0; q < 5; ++q) F[q] = fl[q];
        return;
    }
    if (sr <= T(0)) {
#pragma unroll
        for (int q = 0; q < 5; ++q) F[q] = fr[q];
        return;
    }
    const T dl = wl[0] * (sl - unl);
    const T dr = wr[0] * (sr - unr);
    const T ss = ((wr[4] - wl[4]) + (unl * dl - unr * dr)) / (dl - dr);
    const bool left = ss >= T(0);
    T w[5], u[5], f[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        w[q] = left ? wl[q] : wr[q];
        u[q] = left ? ul[q] : ur[q];
        f[q] = left ? fl[q] : fr[q];
    }
    const T sk = left ? sl : sr;
    const T dk = left ? dl : dr;
    const T fac = dk / (sk - ss);
    T us[5];
    us[0] = fac;
    us[1] = fac * w[1];
    us[2] = fac * w[2];
    us[3] = fac * w[3];
    us[1 + D] = fac * ss;
    us[4] = fac * (u[4] / w[0] + (ss - w[1 + D]) * (ss + w[4] / dk));
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = f[q] + sk * (us[q] - u[q]);
}

// flux through the face between cells c1 and c2 of the four consecutive staged cells c0..c3 (component stride
// PCELLS): minmod-limited left and right states, then HLLC along axis D
template <typename T, int D>
__device__ __forceinline__ void flux4(const Gas<T>& G, const T* c0, const T* c1, const T* c2, const T* c3, T F[5]) {
    T wl[5], wr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T a = c0[q * PCELLS], b = c1[q * PCELLS], c = c2[q * PCELLS], d = c3[q * PCELLS];
        wl[q] = b + T(0.5) * minmod(b - a, c - b);
        wr[q] = c - T(0.5) * minmod(c - b, d - c);
    }
    hllc<T, D>(G, wl, wr, F);
}

// stage plane p (clamped into the grid: the outgoing boundary's zero-gradient ghosts) of the column at (i0, j0)
template <typename T>
__device__ __forceinline__ void stage_plane(T (*ws)[PCELLS], const StageArgs<T>& a, int i0, int j0, int p) {
    const int kk = min(max(p, 0), a.nz - 1);
    for (int c = threadIdx.x; c < PCELLS; c += NT) {
        const int lx = c % PX, ly = c / PX;
        const int i = min(max(i0 - HALO + lx, 0), a.nx - 1);
        const int j = min(max(j0 - HALO + ly, 0), a.ny - 1);
        const long long o = ((long long)kk * a.ny + j) * a.nx + i;
        T u[5], w[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = __ldg(a.Uin + q * a.n + o);
        cons_to_prim(a.gas.gm1, u, w);
#pragma unroll
        for (int q = 0; q < 5; ++q) ws[q][c] = w[q];
    }
}

template <typename T>
__device__ __forceinline__ void apply_floors(const Gas<T>& G, T u[5]) {
    if (u[0] < G.rho_floor) u[0] = G.rho_floor;
    T vx, vy, vz;
    const T ke = kinetic(u, vx, vy, vz);
    const T p = G.gm1 * (u[4] - ke);
    if (p < G.p_floor) u[4] = G.p_floor / G.gm1 + ke;
}

// One Runge-Kutta stage: STAGE 1 writes u0 + dt L(u0); STAGE 2 writes (u0 + (u1 + dt L(u1))) / 2.
template <typename T, int STAGE>
__global__ void __launch_bounds__(NT, sizeof(T) == 8 ? 2 : 3) k_hydro_stage(StageArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smraw);
    const int tid = threadIdx.x, tx = tid & (TX - 1), ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int k0 = blockIdx.z * a.zb, k1 = min(a.nz, k0 + a.zb);
    const int i = i0 + tx, j = j0 + ty;
    const bool own = i < a.nx && j < a.ny;
    const int cc = (ty + HALO) * PX + tx + HALO;  // this thread's cell in a staged plane
    const Gas<T> G = a.gas;

    for (int p = k0 - 2; p <= k0 + 1; ++p) stage_plane(sm.w[slot(p)], a, i0, j0, p);
    __syncthreads();
    T fzl[5], fzh[5];
    flux4<T, 2>(G, &sm.w[slot(k0 - 2)][0][cc], &sm.w[slot(k0 - 1)][0][cc], &sm.w[slot(k0)][0][cc],
                &sm.w[slot(k0 + 1)][0][cc], fzl);
    __syncthreads();  // plane k0-2's slot is refilled next

    for (int k = k0; k < k1; ++k) {
        T u[5], u0[5], acc[3];
        const long long o = ((long long)k * a.ny + (own ? j : 0)) * a.nx + (own ? i : 0);
        if (own) {
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = __ldg(a.Uin + q * a.n + o);
            if (STAGE == 2) {
#pragma unroll
                for (int q = 0; q < 5; ++q) u0[q] = a.U0[q * a.n + o];
            }
            if (a.A) {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[q] = __ldg(a.A + q * a.n + o);
            }
        }
        stage_plane(sm.w[slot(k + 2)], a, i0, j0, k + 2);
        __syncthreads();
        const T(*W)[PCELLS] = sm.w[slot(k)];
        for (int f = tid; f < NXF; f += NT) {
            const int row = f / (TX + 1), af = f - row * (TX + 1);
            const int c0 = (row + HALO) * PX + af;  // cells af-2 .. af+1 of the row: the face between af-1 and af
            T F[5];
            flux4<T, 0>(G, &W[0][c0], &W[0][c0 + 1], &W[0][c0 + 2], &W[0][c0 + 3], F);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.fx[q][f] = F[q];
        }
        for (int f = tid; f < NYF; f += NT) {
            const int fj = f / TX, col = f - fj * TX;
            const int c0 = fj * PX + col + HALO;  // rows fj-2 .. fj+1 of the column: the face between fj-1 and fj
            T F[5];
            flux4<T, 1>(G, &W[0][c0], &W[0][c0 + PX], &W[0][c0 + 2 * PX], &W[0][c0 + 3 * PX], F);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.fy[q][f] = F[q];
        }
        flux4<T, 2>(G, &sm.w[slot(k - 1)][0][cc], &sm.w[slot(k)][0][cc], &sm.w[slot(k + 1)][0][cc],
                    &sm.w[slot(k + 2)][0][cc], fzh);
        __syncthreads();
        if (own) {
            T r[5], un[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                r[q] = sm.fx[q][ty * (TX + 1) + tx] - sm.fx[q][ty * (TX + 1) + tx + 1];
                r[q] = r[q] + (sm.fy[q][ty * TX + tx] - sm.fy[q][(ty + 1) * TX + tx]);
                r[q] = r[q] + (fzl[q] - fzh[q]);
                r[q] = r[q] * a.inv_h;
            }
            if (a.A) {
                r[1] = r[1] + u[0] * acc[0];
                r[2] = r[2] + u[0] * acc[1];
                r[3] = r[3] + u[0] * acc[2];
                r[4] = r[4] + ((u[1] * acc[0] + u[2] * acc[1]) + u[3] * acc[2]);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (STAGE == 1) un[q] = u[q] + a.dt * r[q];
                else un[q] = T(0.5) * (u0[q] + (u[q] + a.dt * r[q]));
            }
            apply_floors(G, un);
#pragma unroll
            for (int q = 0; q < 5; ++q) a.Uout[q * a.n + o] = un[q];
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) fzl[q] = fzh[q];
    }
}

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

// per-block partial sums over the bound cells (E + rho phi < 0), in FP64 from the state's values
template <typename T>
__global__ void __launch_bounds__(hg::kRedThreads) k_virial(const T* __restrict__ U, const double* __restrict__ phi,
                                                           long long n, double* __restrict__ red) {
    __shared__ double sh[32];
    double acc[kVirialSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        double u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = (double)U[q * n + c];
        if (u[0] > acc[4]) acc[4] = u[0];
        const double rp = u[0] * phi[c];
        if (u[4] + rp < 0.0) {
            double vx, vy, vz;
            const double ke = kinetic(u, vx, vy, vz);
            acc[0] += rp;
            acc[1] += u[4] - ke;
            acc[2] += ke;
            acc[3] += u[0];
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

template <typename T>
int launch_stage(hg_hydro* H, int stage, const void* Uin, const void* U0, const void* A, void* Uout, double dt) {
    static unsigned long long attr_done[2] = {0, 0};
    StageArgs<T> a;
    a.Uin = (const T*)Uin;
    a.U0 = (const T*)U0;
    a.A = (const T*)A;
    a.Uout = (T*)Uout;
    a.n = H->n;
    a.nx = H->nx;
    a.ny = H->ny;
    a.nz = H->nz;
    a.zb = stage_zb(H);
    a.dt = (T)dt;
    a.inv_h = (T)(1.0 / H->h);
    a.gas.gamma = (T)H->gamma;
    a.gas.gm1 = (T)(H->gamma - 1.0);
    a.gas.rho_floor = (T)H->rho_floor;
    a.gas.p_floor = (T)H->p_floor;
    const int smem = (int)sizeof(Smem<T>);
    dim3 grid((H->nx + TX - 1) / TX, (H->ny + TY - 1) / TY, (H->nz + a.zb - 1) / a.zb);
    int rc;
    if (stage == 1) {
        if ((rc = hg::smem_attr_once((const void*)k_hydro_stage<T, 1>, smem, &attr_done[0]))) return rc;
        k_hydro_stage<T, 1><<<grid, NT, smem, H->stream>>>(a);
    } else {
        if ((rc = hg::smem_attr_once((const void*)k_hydro_stage<T, 2>, smem, &attr_done[1]))) return rc;
        k_hydro_stage<T, 2><<<grid, NT, smem, H->stream>>>(a);
    }
    HH_LAUNCHED("k_hydro_stage");
    return HG_OK;
}

int launch_stage_any(hg_hydro* H, int stage, const void* Uin, const void* U0, const void* A, void* Uout, double dt) {
    return H->dtype == HG_DT_F64 ? launch_stage<double>(H, stage, Uin, U0, A, Uout, dt)
                                 : launch_stage<float>(H, stage, Uin, U0, A, Uout, dt);
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
}

}  // namespace

extern "C" {

int hg_hydro_init(hg_hydro** out, int nx, int ny, int nz, double h, double gamma, double rho_floor, double p_floor,
                  int dtype, void* cuda_stream) {
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
    if (!H || !n) return fail(HG_ERR_ARG, "null argument");
    *n = H->launches;
    return HG_OK;
}

void hg_hydro_free(hg_hydro* H) {
    if (!H) return;
    cudaSetDevice(H->device);
    cudaStreamSynchronize(H->stream);
    release(H);
    delete H;
}

}  // extern "C"
