// The TMA-staged compensated-float sweep of one tile (used by the single-grid kernel in stencil_tma.cu and by the
// batched launch in stencil.cu), with its shared-memory stage geometry and the mbarrier / bulk-tensor-copy helpers.
//
// A block owns a tile of 128 x-cells x WY rows and marches in z through a chunk of planes.  One producer warp
// streams the planes of the chunk into a ring of S shared-memory stages with cp.async.bulk.tensor (TMA): per plane
// the hi and lo-code rows j0-1 .. j0+WY (the y halo) over cells x0-4 .. x0+131 (a 16-byte-aligned start that
// includes the x halo), and the dlt and s rows of the tile.  WY consumer warps (one row each, 4 cells per lane)
// wait on a stage's mbarrier, read their row and its y neighbours from shared memory, keep the -z/centre planes of
// their own row in registers, take x neighbours by warp shuffles, and store hi', lo', dlt' straight to global
// memory; each consumer warp then releases the stage on its "empty" mbarrier.  The memory-level parallelism is set
// by the S - 2 planes the producer keeps in flight, not by how long the consumers take per plane.
//
// HBM bytes per cell: 24 (read hi 4, lo code 2, dlt 4, s 4; write hi 4, lo 2, dlt 4), plus the y-halo rows and the
// z-halo plane of each block, mostly served by L2.  Every wait is bounded in time: a wait that gives up sets the
// grid's error word (reported as HG_ERR_TIMEOUT by the host) and ends the warp's work without leaving any thread
// of the block waiting.
#pragma once

#include <cuda.h>
#include <cuda_pipeline.h>

#include "cell.cuh"
#include "hg_internal.cuh"
#include "sweep_f32k.cuh"

namespace hg {

constexpr int kTX = 128;                // cells of a tile row
constexpr int kHX = kTX + 8;            // hi / lo-code row of a stage: cells x0-4 .. x0+131
constexpr int kTmaWY = 8;               // rows per block (consumer warps)
constexpr int kStages = 4;              // shared-memory ring depth
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound on any single wait: 1 s

__host__ __device__ constexpr int align128(int b) { return (b + 127) / 128 * 128; }

template <int WY>
struct StageGeom {
    static constexpr int hrows = WY + 2;
    static constexpr int h_tx = hrows * kHX * 4;  // bytes the TMA delivers
    static constexpr int l_tx = hrows * kHX * 2;
    static constexpr int d_tx = WY * kTX * 4;
    static constexpr int h_off = 0;
    static constexpr int l_off = align128(h_tx);
    static constexpr int d_off = l_off + align128(l_tx);
    static constexpr int r_off = d_off + d_tx;
    static constexpr int bytes = r_off + d_tx;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity to complete; false (and the error word set) after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity, int* err,
                                          unsigned long long limit_ns = kWaitNs) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (!mbar_test(bar, parity)) {
        if (now_ns() - t0 > limit_ns) {
            atomicOr(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ uint2 ldsl4(const lo_t* p) { return *reinterpret_cast<const uint2*>(p); }

// The sweep of tile (bx, by) and z chunk bz of one grid by a block of 32 (WY + 1) threads (flat thread index),
// with the stage ring in `smem` and 2 S mbarriers in `bars`.  m_hi .. m_s: tensor maps of hi, lo codes, dlt and s
// of level n (kernel parameters or global memory).  With B.periodic set (batched launches) the consumers also copy
// their tile's new boundary values into the periodic ghosts after the march.
template <int WY, int S>
__device__ __forceinline__ void tma_sweep(const CUtensorMap* m_hi, const CUtensorMap* m_lo, const CUtensorMap* m_d,
                                          const CUtensorMap* m_s, const SweepArgs& A, int bx, int by, int bz,
                                          int* err, unsigned char* smem, unsigned long long* bars) {
    using G = StageGeom<WY>;
    unsigned long long* bar_full = bars;
    unsigned long long* bar_empty = bars + S;
    const Layout& L = A.L;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int x0 = bx * kTX, j0 = by * WY;
    const int k0 = bz * A.zb, k1 = min(L.nz, k0 + A.zb);
    const int planes = k1 - k0 + 1;  // planes k0 .. k1 are staged (plane k1 only as the +z neighbour: hi, lo)

    // Robin grids: the producer warp also writes the x- and y-face ghosts of level n+1 that border this tile (from
    // the staged level-n values, some planes behind its copies), so that this serial work never delays a consumer;
    // the consumers of the first and last chunk write the z-face ghosts once, before and after their march
    const Bnd& B = A.B;
    const bool fx0 = B.faces && bx == 0, fx1 = B.faces && bx == (int)A.gx - 1;
    const bool fy0 = B.faces && by == 0, fy1 = B.faces && by == (int)A.gy - 1;
    const bool faces = fx0 || fx1 || fy0 || fy1;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_addr(&bar_full[s]), 1);
            mbar_init(smem_addr(&bar_empty[s]), WY + (faces ? 1 : 0));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (warp == WY) {  // producer
        constexpr int lag = S - 1;  // face work trails the copies by this many planes
        float* hi_n = (float*)A.hi_n;
        lo_t* lo_n = (lo_t*)A.lo_n;
        // face-ghost lanes: x faces -- lanes 0..WY-1 the rows of face -x, lanes 16..16+WY-1 those of face +x;
        // y faces -- every lane 4 ghosts of row -1 (first row of tiles) and/or row ny (last row of tiles)
        const int w = lane & 15, side = lane >> 4, jx = j0 + w;
        const bool xlane = w < WY && jx < L.ny && (side ? fx1 : fx0);
        // Robin coefficients: the x-face ones travel to shared memory by asynchronous copies issued with each plane's
        // bulk copies (`lag` planes before they are used, so their latency never reaches this warp); the y-face ones
        // (first and last row of tiles only) are loaded one face plane ahead into registers
        __shared__ float2 cxs[S][32];
        float2 cy[2][4];
        auto load_coef = [&](int k) {
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = x0 + 4 * lane + e;
                    cy[s2][e] = (s2 ? fy1 : fy0) && i < L.nx ? B.robin32[B.off[2 + s2] + (long long)k * L.nx + i]
                                                              : make_float2(0.f, 0.f);
                }
        };
        if (faces) load_coef(k0);
        int issued = 0;
        bool ok = true;
        for (int it = 0; it < planes + (faces ? lag : 0) && ok; ++it) {
            if (it < planes) {
                if (lane == 0) {
                    const int s = it % S, p = k0 + it;
                    if (it >= S) ok = mbar_wait(smem_addr(&bar_empty[s]), (unsigned)((it / S - 1) & 1), err);
                    if (ok) {
                        const uint32_t full = smem_addr(&bar_full[s]);
                        unsigned char* st = smem + s * G::bytes;
                        const bool body = p < k1;
                        mbar_expect_tx(full, G::h_tx + G::l_tx + (body ? 2 * G::d_tx : 0));
                        tma_load_3d(smem_addr(st + G::h_off), m_hi, x0, j0, p + 1, full);
                        tma_load_3d(smem_addr(st + G::l_off), m_lo, x0, j0, p + 1, full);
                        if (body) {
                            tma_load_3d(smem_addr(st + G::d_off), m_d, x0 + 4, j0 + 1, p + 1, full);
                            tma_load_3d(smem_addr(st + G::r_off), m_s, x0 + 4, j0 + 1, p + 1, full);
                        }
                        issued = it + 1;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                issued = __shfl_sync(0xffffffffu, issued, 0);
            }
            if (faces) {  // one copy group per iteration (empty when there is nothing to copy), so counts stay uniform
                if (xlane && it < planes - 1)
                    __pipeline_memcpy_async(&cxs[it % S][lane], &B.robin32[B.off[side] + (long long)(k0 + it) * L.ny + jx],
                                            sizeof(float2));
                __pipeline_commit();
            }
            const int pf = it - lag;  // plane (chunk-relative) whose face ghosts are due; the chunk's own planes only
            if (faces && ok && pf >= 0 && pf < planes - 1) {
                const int s = pf % S, k = k0 + pf;
                __pipeline_wait_prior(lag);  // the copy group of plane pf has landed
                const float2 ax = cxs[s][lane];
                float2 ay[2][4];
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
                    for (int e = 0; e < 4; ++e) ay[s2][e] = cy[s2][e];
                if (pf + 1 < planes - 1) load_coef(k + 1);
                if (!(ok = mbar_wait(smem_addr(&bar_full[s]), (unsigned)((pf / S) & 1), err))) break;
                const float* H = (const float*)(smem + s * G::bytes + G::h_off);
                const lo_t* Lo = (const lo_t*)(smem + s * G::bytes + G::l_off);
                if (xlane) {
                    const int tg = side ? L.nx - x0 + 4 : 3, ti = side ? tg - 1 : 4;  // stage elements
                    const int row = (w + 1) * kHX;
                    const float hg = H[row + tg], hin = H[row + ti];
                    float gh, gl;
                    robin_update_f32k(ax.x, ax.y, hg, lo_decode(hg, Lo[row + tg]), hin, lo_decode(hin, Lo[row + ti]),
                                      gh, gl);
                    const long long q = L.at(side ? L.nx : -1, jx, k);
                    if (idx_ok(q, 1, L.elems, B.err)) {
                        hi_n[q] = gh;
                        lo_n[q] = lo_encode(gh, gl);
                    }
                }
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    if (!(s2 ? fy1 : fy0)) continue;
                    const int rg = s2 ? L.ny - j0 + 1 : 0, ri = s2 ? rg - 1 : 1;  // stage rows
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = x0 + 4 * lane + e;
                        if (i < L.nx) {
                            const int t = 4 + 4 * lane + e;
                            const float hg = H[rg * kHX + t], hin = H[ri * kHX + t];
                            float gh, gl;
                            robin_update_f32k(ay[s2][e].x, ay[s2][e].y, hg, lo_decode(hg, Lo[rg * kHX + t]), hin,
                                              lo_decode(hin, Lo[ri * kHX + t]), gh, gl);
                            const long long q = L.at(i, s2 ? L.ny : -1, k);
                            if (idx_ok(q, 1, L.elems, B.err)) {
                                hi_n[q] = gh;
                                lo_n[q] = lo_encode(gh, gl);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&bar_empty[s]));
            }
        }
        // the copies still in flight belong to the last S issued stages; make sure they have landed before the block
        // can end (they have, unless a consumer gave up early)
        if (lane == 0)
            for (int it = issued - S > 0 ? issued - S : 0; it < issued; ++it)
                mbar_wait(smem_addr(&bar_full[it % S]), (unsigned)((it / S) & 1), err);
        return;
    }

    // consumers: warp w owns row j = j0 + w, lane owns cells i0 .. i0 + 3
    const float nu2 = A.nu2f;
    const int j = j0 + warp;
    const int i0 = x0 + lane * 4;
    const bool active = i0 < L.nx && j < L.ny;
    const float* __restrict__ hi_c = (const float*)A.hi_c;
    const lo_t* __restrict__ lo_c = (const lo_t*)A.lo_c;
    float* __restrict__ hi_n = (float*)A.hi_n;
    lo_t* __restrict__ lo_n = (lo_t*)A.lo_n;
    float* __restrict__ dlt = (float*)A.dlt;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int hrow = (warp + 1) * kHX + 4 + 4 * lane;  // this lane's group in a stage's hi / lo rows
    long long q = L.at(i0, j, k0);

    // plane k0 - 1 of the own row straight from global memory (it is not staged)
    float4 hm = z4, lm = z4;
    if (i0 <= L.nx && j < L.ny) {
        hm = __ldg(reinterpret_cast<const float4*>(hi_c + q - L.plane));
        lm = lo_decode4(hm, __ldg(reinterpret_cast<const uint2*>(lo_c + q - L.plane)));
    }
    // a wait that gives up ends this warp's march, but not before the epilogue barrier (no thread is left waiting)
    bool ok = mbar_wait(smem_addr(&bar_full[0]), 0u, err);
    float4 hc = lds4((const float*)(smem + G::h_off) + hrow);
    float4 lc = lo_decode4(hc, ldsl4((const lo_t*)(smem + G::l_off) + hrow));
    // Robin z faces, by the blocks of the first and last chunk: ghost plane -1 from (plane -1, plane 0), ghost
    // plane nz from (plane nz, plane nz - 1), for this lane's 4 cells
    auto zface = [&](int f, const float4& hg, const float4& lg, const float4& hin, const float4& lin, long long qg) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (i0 + e < L.nx) {
                const float2 ab = B.robin32[B.off[f] + (long long)j * L.nx + i0 + e];
                float gh, gl;
                robin_update_f32k(ab.x, ab.y, el(hg, e), el(lg, e), el(hin, e), el(lin, e), gh, gl);
                if (!idx_ok(qg + e, 1, L.elems, B.err)) continue;
                hi_n[qg + e] = gh;
                lo_n[qg + e] = lo_encode(gh, gl);
            }
    };
    if (ok && B.faces && k0 == 0 && active && !(B.zskip & 1)) zface(4, hm, lm, hc, lc, q - L.plane);

    for (int it = 0; it < planes - 1 && ok; ++it) {
        const int sc = it % S, sn = (it + 1) % S;
        if (!(ok = mbar_wait(smem_addr(&bar_full[sn]), (unsigned)(((it + 1) / S) & 1), err))) break;
        const unsigned char* cur = smem + sc * G::bytes;
        const unsigned char* nxt = smem + sn * G::bytes;
        const float* Hc = (const float*)(cur + G::h_off);
        const lo_t* Lc = (const lo_t*)(cur + G::l_off);
        const float4 hp = lds4((const float*)(nxt + G::h_off) + hrow);
        const float4 lp = lo_decode4(hp, ldsl4((const lo_t*)(nxt + G::l_off) + hrow));
        const float4 hs = lds4(Hc + hrow - kHX), hn = lds4(Hc + hrow + kHX);
        const float4 ls = lo_decode4(hs, ldsl4(Lc + hrow - kHX)), ln = lo_decode4(hn, ldsl4(Lc + hrow + kHX));
        const float4 d = lds4((const float*)(cur + G::d_off) + warp * kTX + 4 * lane);
        const float4 r = lds4((const float*)(cur + G::r_off) + warp * kTX + 4 * lane);
        float hl = __shfl_up_sync(0xffffffffu, hc.w, 1), ll = __shfl_up_sync(0xffffffffu, lc.w, 1);
        float hr = __shfl_down_sync(0xffffffffu, hc.x, 1), lr = __shfl_down_sync(0xffffffffu, lc.x, 1);
        if (lane == 0) {
            hl = Hc[hrow - 1];
            ll = lo_decode(hl, Lc[hrow - 1]);
        }
        if (lane == 31) {
            hr = Hc[hrow + 4];
            lr = lo_decode(hr, Lc[hrow + 4]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bar_empty[sc]));  // this warp is done with plane k's stage
        if (active)
            group_update_store(L, B, nu2, i0, q, hc, lc, hl, ll, hr, lr, hs, hn, ls, ln, hm, hp, lm, lp, d, r,
                               hi_n, lo_n, dlt);
        hm = hc;
        hc = hp;
        lm = lc;
        lc = lp;
        q += L.plane;
    }
    if (ok && B.faces && k1 == L.nz && active && !(B.zskip & 2))
        zface(5, hc, lc, hm, lm, q);  // hc: plane nz, hm: plane nz - 1
    if (B.periodic) {  // batched launches: periodic ghosts of the tile's boundary cells, after all consumers stored
        asm volatile("bar.sync 1, %0;" ::"r"(32 * WY) : "memory");
        if (ok)
            block_periodic_copies(L, x0, j0, WY, k0, k1, bx, by, A.gx, A.gy, tid, 32 * WY,
                                  [&](long long qs, long long qd) {
                                      if (!idx_ok(qd, 1, L.elems, B.err)) return;
                                      hi_n[qd] = hi_n[qs];
                                      lo_n[qd] = lo_n[qs];
                                  });
    }
}

}  // namespace hg
