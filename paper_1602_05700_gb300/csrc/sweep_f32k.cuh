// Pieces of the compensated-float sub-step shared by the register-staged sweep (stencil.cu, also the batched
// launch) and the TMA-staged sweep (stencil_tma.cu): a lane's 4-cell group update, its stores, and the periodic
// x-face ghosts of the new level.  Both sweeps thereby compute and store bit-identical results.
#pragma once

#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

__device__ __forceinline__ float el(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ void set(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

// One lane's 4 consecutive cells i0..i0+3 of row j, plane k: c/lc the level-n values of the group, hl/ll and hr/lr
// its x neighbours (cells i0-1 and i0+4), hs/hn (ls/ln) the -y/+y rows, hm/hp (lm/lp) the -z/+z planes, d the
// increments, r the source.  Stores hi', lo' (coded), dlt' at padded index q (cells beyond nx are not stored) and,
// for periodic grids whose x-face ghosts are produced in the sweep, the ghost copies of cells 0 and nx-1.
__device__ __forceinline__ void group_update_store(const Layout& L, const Bnd& B, float nu2, int i0, long long q,
                                                   const float4& hc, const float4& lc, float hl, float ll,
                                                   float hr, float lr, const float4& hs, const float4& hn,
                                                   const float4& ls, const float4& ln, const float4& hm,
                                                   const float4& hp, const float4& lm, const float4& lp,
                                                   const float4& d, const float4& r, float* __restrict__ hi_n,
                                                   lo_t* __restrict__ lo_n, float* __restrict__ dlt) {
    float4 ho, lo, dout;
    f32k_update4_scalar(hc, lc, hl, ll, hr, lr, hs, hn, hm, hp, ls, ln, lm, lp, d, r, nu2, ho, lo, dout);
    if (!idx_ok(q, 4, L.elems, B.err)) return;
    if (i0 + 3 < L.nx) {
        *reinterpret_cast<float4*>(hi_n + q) = ho;
        *reinterpret_cast<uint2*>(lo_n + q) = lo_encode4(ho, lo);
        *reinterpret_cast<float4*>(dlt + q) = dout;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (i0 + e < L.nx) {
                hi_n[q + e] = el(ho, e);
                lo_n[q + e] = lo_encode(el(ho, e), el(lo, e));
                dlt[q + e] = el(dout, e);
            }
    }
    // periodic x-face ghosts of level n+1 (copies of the new values at the opposite face), by the two lanes that
    // hold the face cells: the ghosts lie in the same rows, so these are the only scattered stores
    if (B.xfaces == HG_BC_PERIODIC) {
        const int elast = L.nx - 1 - i0;  // element holding cell nx-1, if 0..3
        if (i0 == 0 && idx_ok(q + L.nx, 1, L.elems, B.err)) {
            hi_n[q + L.nx] = ho.x;
            lo_n[q + L.nx] = lo_encode(ho.x, lo.x);
        }
        if (elast >= 0 && elast < 4 && idx_ok(q + elast - L.nx, 1, L.elems, B.err)) {
            hi_n[q + elast - L.nx] = el(ho, elast);
            lo_n[q + elast - L.nx] = lo_encode(el(ho, elast), el(lo, elast));
        }
    }
}

__device__ __forceinline__ int block_tid() { return threadIdx.y * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int block_nth() { return blockDim.x * blockDim.y; }

// Periodic boundaries: after its own sweep (and a barrier among the threads that wrote it, so that they see each
// other's stores), a block copies the new values of its cells on a face into the ghosts of the opposite face, with
// threads tid = 0 .. nth-1.  copy(src, dst) takes padded indices; each boundary cell belongs to exactly one block.
template <class Copy>
__device__ __forceinline__ void block_periodic_copies(const Layout& L, int x0, int j0, int wy, int k0, int k1, int bx,
                                                      int by, int gx, int gy, int tid, int nth, Copy&& copy,
                                                      int tw = 128) {
    const int jn = min(wy, L.ny - j0), xn = min(tw, L.nx - x0), kn = k1 - k0;
    const long long wx = L.nx, wy_ = (long long)L.ny * L.pitch, wz = (long long)L.nz * L.plane;
    if (bx == 0)
        for (int t = tid; t < jn * kn; t += nth) {
            const long long q = L.at(0, j0 + t % jn, k0 + t / jn);
            copy(q, q + wx);
        }
    if (bx == gx - 1)
        for (int t = tid; t < jn * kn; t += nth) {
            const long long q = L.at(L.nx - 1, j0 + t % jn, k0 + t / jn);
            copy(q, q - wx);
        }
    if (by == 0)
        for (int t = tid; t < xn * kn; t += nth) {
            const long long q = L.at(x0 + t % xn, 0, k0 + t / xn);
            copy(q, q + wy_);
        }
    if (by == gy - 1)
        for (int t = tid; t < xn * kn; t += nth) {
            const long long q = L.at(x0 + t % xn, L.ny - 1, k0 + t / xn);
            copy(q, q - wy_);
        }
    if (k0 == 0)
        for (int t = tid; t < xn * jn; t += nth) {
            const long long q = L.at(x0 + t % xn, j0 + t / xn, 0);
            copy(q, q + wz);
        }
    if (k1 == L.nz)
        for (int t = tid; t < xn * jn; t += nth) {
            const long long q = L.at(x0 + t % xn, j0 + t / xn, L.nz - 1);
            copy(q, q - wz);
        }
}

}  // namespace hg
