// Device code of the ideal-gas hydrodynamics (include/hg_hydro.h), included by hydro.cu (the FP64 instance and the
// reductions, compiled without multiply-add contraction) and hydro_f32.cu (the FP32 stage kernel, compiled with
// contraction and approximate division and square root).  Everything here has internal linkage, so each
// translation unit keeps its own instance with its own floating-point flags.
//
// Scheme (paper Sec. 2; the library's reading, fixed by the ABI header): piecewise-linear primitives with
// monotonized-central limited slopes, HLLC fluxes with Davis' wave-speed bounds, outgoing (zero-gradient) boundaries, two-stage SSP
// Runge-Kutta with the gravity source (0, rho a, m . a), floors after each stage.
//
// Kernel design (one launch per Runge-Kutta stage): a block owns a 32 x 8 column of cells and marches along z
// through a chunk of planes.  A ring of primitive planes (the column plus a 2-cell halo in x and y) sits in
// shared memory; each plane of the global state is read once per block and converted to primitives once (its
// loads are issued before the current plane's face fluxes and consumed after them).  Every face flux is evaluated
// once: the 33 x 8 x-faces and 32 x 9 y-faces of the current plane are computed by the block's threads in two full
// rounds and one round of two warps, into shared memory; the z-face above each cell is kept in registers and
// becomes the next plane's lower face, and the z-slope of its upper cell is kept for the next z-face.  The update,
// the gravity source, the stage combination and the floors are fused into the same pass, so a stage reads the
// stage state (and, for stage 2, the step's initial state and a) once and writes the new state once.
#pragma once

#include <cuda_runtime.h>

namespace hg {

// one Runge-Kutta stage launch (stage 1: Uout = Uin + dt L(Uin); stage 2: Uout = (U0 + (Uin + dt L(Uin))) / 2)
struct HydroStageLaunch {
    cudaStream_t stream;
    int nx, ny, nz, zb, stage;
    long long n;
    double h, gamma, rho_floor, p_floor, dt;
    const void* Uin;
    const void* U0;
    const void* A;  // acceleration planes or null
    void* Uout;
};
cudaError_t hydro_stage_f64(const HydroStageLaunch& L);  // hydro.cu
cudaError_t hydro_stage_f32(const HydroStageLaunch& L);  // hydro_f32.cu

}  // namespace hg

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO, PCELLS = PX * PY;  // 36 x 12 cells per staged plane
constexpr int NXF = (TX + 1) * TY;  // x-faces of one plane of the column
constexpr int NYF = TX * (TY + 1);  // y-faces

// division and square root: exact (IEEE round-to-nearest) in FP64, the reference mode; the hardware's approximate
// reciprocal-based division and square root in FP32, whose results are compared within tolerance anyway
__device__ __forceinline__ double hdiv(double a, double b) { return a / b; }
__device__ __forceinline__ double hsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float hdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float hsqrt(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Shared-memory ring of staged planes.  FP32: five planes and double-buffered face fluxes, so one barrier per plane
// suffices (plane k+2 is staged and the x/y-faces of plane k computed before it; the z-face and the update after
// it).  FP64: four planes and one face buffer (the smaller footprint keeps two blocks per SM), two barriers per plane.
template <typename T>
struct Ring {
    static constexpr int planes = sizeof(T) == 4 ? 5 : 4;
    static constexpr int bufs = planes == 5 ? 2 : 1;
    static constexpr bool one_barrier = planes == 5;
    __device__ static __forceinline__ int slot(int p) { return (p + 2 * planes) % planes; }  // p >= -2
};

template <typename T>
struct Smem {
    T w[Ring<T>::planes][5][PCELLS];  // primitive planes, ring by plane index
    T fx[Ring<T>::bufs][5][NXF];
    T fy[Ring<T>::bufs][5][NYF];
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


template <typename T>
__device__ __forceinline__ T kinetic(const T u[5], T& vx, T& vy, T& vz) {
    vx = hdiv(u[1], u[0]);
    vy = hdiv(u[2], u[0]);
    vz = hdiv(u[3], u[0]);
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
    u[4] = hdiv(w[4], gm1) + T(0.5) * w[0] * ((w[1] * w[1] + w[2] * w[2]) + w[3] * w[3]);
}

// minmod: the smaller slope in magnitude when both have the same sign, else 0.  FP64 in the comparison form the
// ABI header states; FP32 branch-free as the median of (a, b, 0) (the same value up to the sign of a zero result,
// which no later operation can distinguish except through another zero)
__device__ __forceinline__ double minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}
__device__ __forceinline__ float minmod(float a, float b) {
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));  // the median of (a, b, 0)
}

// half the monotonized-central slope from the one-sided differences a (backward) and b (forward), i.e. the
// reconstruction offset to a face: half of the least-magnitude of 2a, (a + b)/2, 2b when all three have one sign,
// else 0 -- written as minmod((a + b)/4, minmod(a, b)).  Halving is exact, so this selects exactly the value
// 0.5 * mc(a, b) of the three-way form
template <typename T>
__device__ __forceinline__ T mc_half(T a, T b) {
    return minmod(T(0.25) * (a + b), minmod(a, b));
}
// FP32: the same selection as the median of (min, max, 0) of the three candidates (a, b, (a + b)/4), six min/max
// instead of eight
__device__ __forceinline__ float mc_half(float a, float b) {
    const float c = 0.25f * (a + b);
    const float lo = fminf(fminf(a, b), c), hi = fmaxf(fmaxf(a, b), c);
    return fmaxf(lo, fminf(hi, 0.0f));
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

// HLLC flux along axis D between primitive states wl and wr (Davis bounds, Toro-Spruce-Speares star states).
// Only the side the flux is taken from is converted to a conserved state and a physical flux: the left one if
// S_L >= 0, the right one if S_R <= 0 (supersonic: that side's physical flux), else the side of the contact speed's
// sign (F = F_K + S_K (U*_K - U_K)).  Every value is computed by the same operations as a version that evaluates
// both sides and then picks one.
template <typename T, int D>
__device__ __forceinline__ void hllc(const Gas<T>& G, const T wl[5], const T wr[5], T F[5]) {
    const T al = hsqrt(hdiv(G.gamma * wl[4], wl[0]));
    const T ar = hsqrt(hdiv(G.gamma * wr[4], wr[0]));
    const T unl = wl[1 + D], unr = wr[1 + D];
    const T a1 = unl - al, a2 = unr - ar, b1 = unl + al, b2 = unr + ar;
    const T sl = a1 < a2 ? a1 : a2;
    const T sr = b1 > b2 ? b1 : b2;
    const T dl = wl[0] * (sl - unl);
    const T dr = wr[0] * (sr - unr);
    const T ss = hdiv((wr[4] - wl[4]) + (unl * dl - unr * dr), dl - dr);
    const bool upwind = sl >= T(0) || sr <= T(0);
    const bool left = sl >= T(0) || (sr > T(0) && ss >= T(0));
    T w[5], u[5], f[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) w[q] = left ? wl[q] : wr[q];
    const T sk = left ? sl : sr;
    const T dk = left ? dl : dr;
    state_flux<T, D>(G.gm1, w, u, f);
    const T fac = hdiv(dk, sk - ss);
    T us[5];
    us[0] = fac;
    us[1] = fac * w[1];
    us[2] = fac * w[2];
    us[3] = fac * w[3];
    us[1 + D] = fac * ss;
    us[4] = fac * (hdiv(u[4], w[0]) + (ss - w[1 + D]) * (ss + hdiv(w[4], dk)));
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = upwind ? f[q] : f[q] + sk * (us[q] - u[q]);  // a non-finite star value of a
}                                                                                    // supersonic face is never used

// flux through the face between cells c1 and c2 of the four consecutive staged cells c0..c3 (component stride
// PCELLS): MC-limited left and right states, then HLLC along axis D
template <typename T, int D>
__device__ __forceinline__ void flux4(const Gas<T>& G, const T* c0, const T* c1, const T* c2, const T* c3, T F[5]) {
    T wl[5], wr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T a = c0[q * PCELLS], b = c1[q * PCELLS], c = c2[q * PCELLS], d = c3[q * PCELLS];
        wl[q] = b + mc_half(b - a, c - b);
        wr[q] = c - mc_half(c - b, d - c);
    }
    hllc<T, D>(G, wl, wr, F);
}

// z-face between planes k and k+1 of this thread's column: the limited half-slope of plane k (carried from the
// previous plane, where it was the upper cell's) and that of plane k+1 (computed here from planes k, k+1, k+2 and
// carried on); the same operations on the same values as flux4, each slope evaluated once
template <typename T>
__device__ __forceinline__ void zflux(const Gas<T>& G, const T* ck, const T* ck1, const T* ck2, const T sk[5],
                                      T sk1[5], T F[5]) {
    T wl[5], wr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T b = ck[q * PCELLS], c = ck1[q * PCELLS], d = ck2[q * PCELLS];
        sk1[q] = mc_half(c - b, d - c);
        wl[q] = b + sk[q];
        wr[q] = c - sk1[q];
    }
    hllc<T, 2>(G, wl, wr, F);
}

// limited half-slope of this thread's cell in plane p from planes p-1, p, p+1
template <typename T>
__device__ __forceinline__ void zslope(const T* cm, const T* c0, const T* cp, T s[5]) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T a = cm[q * PCELLS], b = c0[q * PCELLS], c = cp[q * PCELLS];
        s[q] = mc_half(b - a, c - b);
    }
}

// Staging of plane p (clamped into the grid: the outgoing boundary's zero-gradient ghosts) of the column at
// (i0, j0), in two halves so that the loads can be issued early and the conversion done later: plane_load reads
// the conserved state of this thread's (at most two) cells of the staged plane into registers, plane_store
// converts them to primitives and writes them to a ring slot.
static_assert(PCELLS <= 2 * NT, "a thread stages at most two cells of a plane");

template <typename T>
struct PlaneRegs {
    T u[2][5];
};

template <typename T>
__device__ __forceinline__ void plane_load(PlaneRegs<T>& r, const StageArgs<T>& a, int i0, int j0, int p) {
    const int kk = min(max(p, 0), a.nz - 1);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int c = threadIdx.x + t * NT;
        if (c < PCELLS) {
            const int lx = c % PX, ly = c / PX;
            const int i = min(max(i0 - HALO + lx, 0), a.nx - 1);
            const int j = min(max(j0 - HALO + ly, 0), a.ny - 1);
            const long long o = ((long long)kk * a.ny + j) * a.nx + i;
#pragma unroll
            for (int q = 0; q < 5; ++q) r.u[t][q] = __ldg(a.Uin + q * a.n + o);
        }
    }
}

template <typename T>
__device__ __forceinline__ void plane_store(T (*ws)[PCELLS], const PlaneRegs<T>& r, T gm1) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int c = threadIdx.x + t * NT;
        if (c < PCELLS) {
            T w[5];
            cons_to_prim(gm1, r.u[t], w);
#pragma unroll
            for (int q = 0; q < 5; ++q) ws[q][c] = w[q];
        }
    }
}

template <typename T>
__device__ __forceinline__ void apply_floors(const Gas<T>& G, T u[5]) {
    if (u[0] < G.rho_floor) u[0] = G.rho_floor;
    T vx, vy, vz;
    const T ke = kinetic(u, vx, vy, vz);
    const T p = G.gm1 * (u[4] - ke);
    if (p < G.p_floor) u[4] = hdiv(G.p_floor, G.gm1) + ke;
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
    using R = Ring<T>;

    for (int p = k0 - 2; p <= k0 + 1; ++p) {
        PlaneRegs<T> pr;
        plane_load(pr, a, i0, j0, p);
        plane_store(sm.w[R::slot(p)], pr, G.gm1);
    }
    __syncthreads();
    T fzl[5], fzh[5], szk[5], szk1[5];  // z-faces below and above plane k; z-slopes of planes k and k+1
    zslope(&sm.w[R::slot(k0 - 2)][0][cc], &sm.w[R::slot(k0 - 1)][0][cc], &sm.w[R::slot(k0)][0][cc], szk);
    zflux(G, &sm.w[R::slot(k0 - 1)][0][cc], &sm.w[R::slot(k0)][0][cc], &sm.w[R::slot(k0 + 1)][0][cc], szk, szk1, fzl);
#pragma unroll
    for (int q = 0; q < 5; ++q) szk[q] = szk1[q];
    if (!R::one_barrier) __syncthreads();  // with four slots, plane k0-2's slot is refilled next

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
        PlaneRegs<T> pr;
        plane_load(pr, a, i0, j0, k + 2);  // with one barrier per plane, converted and stored after the x/y faces
        if (!R::one_barrier) {
            plane_store(sm.w[R::slot(k + 2)], pr, G.gm1);
            __syncthreads();
        }
        const int b = R::one_barrier ? (k & 1) : 0;
        const T(*W)[PCELLS] = sm.w[R::slot(k)];
        // x- and y-faces of plane k: x-face tx of row ty (between cells tx-1 and tx), the y-face below cell
        // (tx, ty), then the last x-face of each row (warp 1, lanes 0-7) and the y-faces above row TY-1 (warp 0)
        {
            T F[5];
            const int c0 = (ty + HALO) * PX + tx;  // cells tx-2 .. tx+1 of row ty
            flux4<T, 0>(G, &W[0][c0], &W[0][c0 + 1], &W[0][c0 + 2], &W[0][c0 + 3], F);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.fx[b][q][ty * (TX + 1) + tx] = F[q];
            const int c1 = ty * PX + tx + HALO;  // rows ty-2 .. ty+1 of column tx
            flux4<T, 1>(G, &W[0][c1], &W[0][c1 + PX], &W[0][c1 + 2 * PX], &W[0][c1 + 3 * PX], F);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.fy[b][q][ty * TX + tx] = F[q];
            if (ty == 0) {
                const int c2 = TY * PX + tx + HALO;  // rows TY-2 .. TY+1: the face between rows TY-1 and TY
                flux4<T, 1>(G, &W[0][c2], &W[0][c2 + PX], &W[0][c2 + 2 * PX], &W[0][c2 + 3 * PX], F);
#pragma unroll
                for (int q = 0; q < 5; ++q) sm.fy[b][q][TY * TX + tx] = F[q];
            } else if (ty == 1 && tx < TY) {
                const int c3 = (tx + HALO) * PX + TX;  // row tx, cells TX-2 .. TX+1: the face between TX-1 and TX
                flux4<T, 0>(G, &W[0][c3], &W[0][c3 + 1], &W[0][c3 + 2], &W[0][c3 + 3], F);
#pragma unroll
                for (int q = 0; q < 5; ++q) sm.fx[b][q][tx * (TX + 1) + TX] = F[q];
            }
        }
        if (!R::one_barrier)
            zflux(G, &sm.w[R::slot(k)][0][cc], &sm.w[R::slot(k + 1)][0][cc], &sm.w[R::slot(k + 2)][0][cc], szk, szk1,
                  fzh);
        else
            plane_store(sm.w[R::slot(k + 2)], pr, G.gm1);
        __syncthreads();
        if (R::one_barrier)
            zflux(G, &sm.w[R::slot(k)][0][cc], &sm.w[R::slot(k + 1)][0][cc], &sm.w[R::slot(k + 2)][0][cc], szk, szk1,
                  fzh);
        if (own) {
            T r[5], un[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                r[q] = sm.fx[b][q][ty * (TX + 1) + tx] - sm.fx[b][q][ty * (TX + 1) + tx + 1];
                r[q] = r[q] + (sm.fy[b][q][ty * TX + tx] - sm.fy[b][q][(ty + 1) * TX + tx]);
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
        for (int q = 0; q < 5; ++q) {
            fzl[q] = fzh[q];
            szk[q] = szk1[q];
        }
    }
}

template <typename T>
cudaError_t launch_hydro_stage(const hg::HydroStageLaunch& L) {
    static unsigned long long attr_done[2] = {0, 0};  // one bit per device, per stage kernel
    StageArgs<T> a;
    a.Uin = (const T*)L.Uin;
    a.U0 = (const T*)L.U0;
    a.A = (const T*)L.A;
    a.Uout = (T*)L.Uout;
    a.n = L.n;
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.zb = L.zb;
    a.dt = (T)L.dt;
    a.inv_h = (T)(1.0 / L.h);
    a.gas.gamma = (T)L.gamma;
    a.gas.gm1 = (T)(L.gamma - 1.0);
    a.gas.rho_floor = (T)L.rho_floor;
    a.gas.p_floor = (T)L.p_floor;
    const int smem = (int)sizeof(Smem<T>);
    const void* fn = L.stage == 1 ? (const void*)k_hydro_stage<T, 1> : (const void*)k_hydro_stage<T, 2>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    unsigned long long& done = attr_done[L.stage == 1 ? 0 : 1];
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done & bit)) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        done |= bit;
    }
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + L.zb - 1) / L.zb);
    if (L.stage == 1) k_hydro_stage<T, 1><<<grid, NT, smem, L.stream>>>(a);
    else k_hydro_stage<T, 2><<<grid, NT, smem, L.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace
