// Two fused sub-steps per HBM round trip (temporal blocking, depth 2) of the compensated-float sub-step, staged by
// TMA (arXiv 1602.05700, Sec. 2: rho is frozen during the wave sub-steps of a hydro step, so consecutive sub-steps
// can be fused without reading the source again).  Dirichlet and Robin grids; periodic grids use temporal.cu.
//
// A block writes a tile of 120 x-cells x 8 rows of level n+2 over a chunk of z planes.  Level n+1 is computed on
// the tile grown by one cell on every side (x0-4 .. x0+123, rows j0-1 .. j0+8: 32 lanes x 4 cells, one warp per
// row, 10 warps), from level n staged with cp.async.bulk.tensor into a ring of 3 shared-memory stages (per plane: hi and lo-code rows j0-2 .. j0+9 over cells x0-12 .. x0+131, dlt and s rows
// j0-1 .. j0+8 over x0-4 .. x0+123).  In z the two levels form a pipeline: the iteration that computes level n+1 at
// plane p (its own row's -z/centre planes in registers, +z and the y rows from the stage) writes that row into a
// 4-slot shared ring, meets the other warps at one named barrier -- after which one thread refills the stage of
// plane p with plane p+3 -- and then computes level n+2 at plane p-1 from the ring (its own rows at planes p-2, p-1,
// the neighbouring rows at p-1) and its level-(n+1) row at p in registers.  Level n+1 is never stored.
//
// Face ghosts at level n+1 follow the boundary condition exactly as a single sweep would write them (Dirichlet: the
// data; Robin: the radiation update from the level-n ghost and its interior neighbour), and the level-(n+2) face
// ghosts that border the tile are written with the new level.  Every level-(n+1) lo goes through the 16-bit code
// (lo_round) as a store and a load would, and all arithmetic is the single sweep's (cell.cuh), so the result is
// bit-identical to two single sweeps.
//
// HBM bytes per cell for the two sub-steps: 24 (read hi, lo, dlt, s; write hi, lo, dlt) plus the halo rows and
// planes of the grown tile, which neighbouring blocks read too (mostly from L2).
#include "sweep_tma.cuh"

namespace hg {

namespace {

constexpr int kOX = 120;          // level-(n+2) cells of a tile row
constexpr int kOW = 8;            // level-(n+2) rows of a tile
constexpr int kR1 = kOW + 2;      // level-(n+1) rows = consumer warps
constexpr int kS2 = 3;            // stage ring depth
constexpr int kRing = 4;          // level-(n+1) ring slots (planes p-2 .. p, and one being refilled)
constexpr int kHX2 = 136;         // staged hi row: cells x0-8 .. x0+127
constexpr int kLX2 = 144;         // staged lo-code row: cells x0-12 .. x0+131 (a 16-byte-aligned start for 2-byte codes)
constexpr int kDX2 = 128;         // staged dlt / s row: cells x0-4 .. x0+123
constexpr int kHR2 = kOW + 4;     // staged hi / lo rows: j0-2 .. j0+9

struct T2 {
    static constexpr int h_tx = kHR2 * kHX2 * 4;
    static constexpr int l_tx = kHR2 * kLX2 * 2;
    static constexpr int d_tx = kR1 * kDX2 * 4;
    static constexpr int h_off = 0;
    static constexpr int l_off = align128(h_tx);
    static constexpr int d_off = l_off + align128(l_tx);
    static constexpr int r_off = d_off + d_tx;
    static constexpr int stage = r_off + d_tx;
    static constexpr int ring_off = kS2 * stage;           // level-(n+1) ring: kRing slots of hi, then of lo
    static constexpr int ring_slot = kR1 * kDX2;           // floats per slot
    static constexpr int smem = ring_off + 2 * kRing * ring_slot * 4;
};

// Robin coefficients (alpha, beta) of a face ghost, or none
__device__ __forceinline__ float2 coef(const Bnd& B, int f, long long t) { return B.robin32[B.off[f] + t]; }

__global__ void __launch_bounds__(32 * kR1, 2)
    k_temporal2_tma(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_lo,
                    const __grid_constant__ CUtensorMap m_d, const __grid_constant__ CUtensorMap m_s,
                    const SweepArgs A, float* __restrict__ d_out, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_full[kS2];
    const Layout& L = A.L;
    const Bnd& B = A.B;
    const bool robin = B.faces != 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kOX, j0 = blockIdx.y * kOW;
    const int k0 = blockIdx.z * A.zb, k1 = min(L.nz, k0 + A.zb);
    const int nload = k1 - k0 + 3;  // level-n planes k0-1 .. k1+1

    // thread 0 issues the copies: the first kS2 planes now, then plane it+kS2 right after the named barrier of
    // iteration it (every warp is done with that stage by then, so no "empty" barrier is needed)
    auto issue = [&](int i) {  // level-n plane k0-1+i into slot i % kS2
        const uint32_t full = smem_addr(&bar_full[i % kS2]);
        unsigned char* st = smem + (i % kS2) * T2::stage;
        const int z = k0 + i;  // padded plane index of plane k0-1+i
        mbar_expect_tx(full, T2::h_tx + T2::l_tx + 2 * T2::d_tx);
        tma_load_3d(smem_addr(st + T2::h_off), &m_hi, x0 - 4, j0 - 1, z, full);
        tma_load_3d(smem_addr(st + T2::l_off), &m_lo, x0 - 8, j0 - 1, z, full);
        tma_load_3d(smem_addr(st + T2::d_off), &m_d, x0, j0, z, full);
        tma_load_3d(smem_addr(st + T2::r_off), &m_s, x0, j0, z, full);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < kS2; ++s) mbar_init(smem_addr(&bar_full[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int i = 0; i < kS2 && i < nload; ++i) issue(i);
    }
    int issued = kS2 < nload ? kS2 : nload;  // tracked by thread 0
    __syncthreads();

    // consumers: warp w computes level n+1 on row j1 = j0-1+w (cells x0-4+4l .. +3) and, for w = 1..8, level n+2 on
    // the same row (lanes 1..30: cells x0 .. x0+119)
    const float nu2 = A.nu2f;
    const int j1 = j0 - 1 + warp;
    const int xa = x0 - 4 + 4 * lane;  // first cell of this lane's group
    const bool row_in = j1 >= 0 && j1 < L.ny;
    const bool row_gy = robin && (j1 == -1 || j1 == L.ny);  // a y-face ghost row
    const bool row_on = j1 >= -1 && j1 <= L.ny;              // a row of the padded array
    float* __restrict__ hi_n = (float*)A.hi_n;
    lo_t* __restrict__ lo_n = (lo_t*)A.lo_n;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float* ring_h = (float*)(smem + T2::ring_off);
    float* ring_l = ring_h + kRing * T2::ring_slot;
    auto ring4 = [&](const float* base, int slot, int off) {
        return *reinterpret_cast<const float4*>(base + slot * T2::ring_slot + off);
    };
    const int hrow = (warp + 1) * kHX2 + 4 + 4 * lane;  // own group in a stage's hi rows
    const int lrow = (warp + 1) * kLX2 + 8 + 4 * lane;  // ... in its lo-code rows
    const int drow = warp * kDX2 + 4 * lane;            // ... in its dlt / s rows, and in a ring slot

    // the class of each of the lane's 4 cells in x: 0 interior, 1 the -x ghost, 2 the +x ghost, 3 elsewhere
    int xc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int x = xa + e;
        xc[e] = (x >= 0 && x < L.nx) ? 0 : x == -1 ? 1 : x == L.nx ? 2 : 3;
    }

    // level n, own row, plane k0-2 (not staged; only needed when k0 > 0)
    float4 hm0 = z4, lm0 = z4;
    if (k0 > 0 && row_on && xa <= L.nx) {
        const long long q = L.at(xa, j1, k0 - 2);
        hm0 = __ldg(reinterpret_cast<const float4*>((const float*)A.hi_c + q));
        lm0 = lo_decode4(hm0, __ldg(reinterpret_cast<const uint2*>((const lo_t*)A.lo_c + q)));
    }
    bool ok = mbar_wait(smem_addr(&bar_full[0]), 0u, err);
    float4 hc0 = lds4((const float*)(smem + T2::h_off) + hrow);
    float4 lc0 = lo_decode4(hc0, ldsl4((const lo_t*)(smem + T2::l_off) + lrow));

    float4 d1c = z4, sc_ = z4;  // level n+1 increments and the source of plane p-1, own row

    const int iters = k1 - k0 + 2;  // level n+1 at planes k0-1 .. k1
    for (int it = 0; it < iters && ok; ++it) {
        const int p = k0 - 1 + it;
        const int si = it % kS2, sn = (it + 1) % kS2;
        if (!(ok = mbar_wait(smem_addr(&bar_full[sn]), (unsigned)(((it + 1) / kS2) & 1), err))) break;
        const unsigned char* cur = smem + si * T2::stage;
        const unsigned char* nxt = smem + sn * T2::stage;
        const float* Hc = (const float*)(cur + T2::h_off);
        const lo_t* Lc = (const lo_t*)(cur + T2::l_off);
        const float4 hp0 = lds4((const float*)(nxt + T2::h_off) + hrow);
        const float4 lp0 = lo_decode4(hp0, ldsl4((const lo_t*)(nxt + T2::l_off) + lrow));
        const float4 hs = lds4(Hc + hrow - kHX2), hn = lds4(Hc + hrow + kHX2);
        const float4 ls = lo_decode4(hs, ldsl4(Lc + lrow - kLX2)), ln = lo_decode4(hn, ldsl4(Lc + lrow + kLX2));
        const float4 d0 = lds4((const float*)(cur + T2::d_off) + drow);
        const float4 s0 = lds4((const float*)(cur + T2::r_off) + drow);
        float hl = __shfl_up_sync(0xffffffffu, hc0.w, 1), ll = __shfl_up_sync(0xffffffffu, lc0.w, 1);
        float hr = __shfl_down_sync(0xffffffffu, hc0.x, 1), lr = __shfl_down_sync(0xffffffffu, lc0.x, 1);
        if (lane == 0) {
            hl = Hc[hrow - 1];
            ll = lo_decode(hl, Lc[lrow - 1]);
        }
        if (lane == 31) {
            hr = Hc[hrow + 4];
            lr = lo_decode(hr, Lc[lrow + 4]);
        }

        // ---- level n+1 at plane p, own row ----
        const bool pl_in = p >= 0 && p < L.nz;
        const bool pl_gz = robin && (p == -1 || p == L.nz);
        float4 h1 = hc0, l1 = lc0, d1 = d0;  // ghosts without an update (Dirichlet data, cells outside) keep level n
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float xl = e == 0 ? hl : el(hc0, e - 1), xr = e == 3 ? hr : el(hc0, e + 1);
            const float lxl = e == 0 ? ll : el(lc0, e - 1), lxr = e == 3 ? lr : el(lc0, e + 1);
            float a = el(hc0, e), b = el(lc0, e), c = el(d0, e);
            if (xc[e] == 0 && row_in && pl_in) {
                f32k_update(xl, xr, el(hs, e), el(hn, e), el(hm0, e), el(hp0, e), el(hc0, e), lxl, lxr, el(ls, e),
                            el(ln, e), el(lm0, e), el(lp0, e), el(lc0, e), el(d0, e), el(s0, e), nu2, a, b, c);
                b = lo_round(a, b);
            } else if (robin) {
                // the face ghosts: exactly one coordinate one cell outside
                int f = -1;
                long long t = 0;
                float gi = 0.f, li = 0.f;
                if (xc[e] != 0 && xc[e] != 3 && row_in && pl_in) {
                    f = xc[e] - 1;
                    t = (long long)p * L.ny + j1;
                    gi = xc[e] == 1 ? xr : xl;
                    li = xc[e] == 1 ? lxr : lxl;
                } else if (xc[e] == 0 && row_gy && pl_in) {
                    f = j1 < 0 ? 2 : 3;
                    t = (long long)p * L.nx + xa + e;
                    gi = j1 < 0 ? el(hn, e) : el(hs, e);
                    li = j1 < 0 ? el(ln, e) : el(ls, e);
                } else if (xc[e] == 0 && row_in && pl_gz) {
                    f = p < 0 ? 4 : 5;
                    t = (long long)j1 * L.nx + xa + e;
                    gi = p < 0 ? el(hp0, e) : el(hm0, e);
                    li = p < 0 ? el(lp0, e) : el(lm0, e);
                }
                if (f >= 0) {
                    const float2 ab = coef(B, f, t);
                    robin_update_f32k(ab.x, ab.y, el(hc0, e), el(lc0, e), gi, li, a, b);
                    b = lo_round(a, b);
                }
            }
            set(h1, e, a);
            set(l1, e, b);
            set(d1, e, c);
        }
        // publish the row (for the neighbouring rows, and as this row's -z / centre planes of the next iterations)
        float* rh = ring_h + (it % kRing) * T2::ring_slot + drow;
        float* rl = ring_l + (it % kRing) * T2::ring_slot + drow;
        *reinterpret_cast<float4*>(rh) = h1;
        *reinterpret_cast<float4*>(rl) = l1;
        asm volatile("bar.sync 2, %0;" ::"r"(32 * kR1) : "memory");
        if (threadIdx.x == 0 && it + kS2 < nload) {  // stage of plane p is free: refill it with plane p+kS2
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(it + kS2);
            issued = it + kS2 + 1;
        }

        // ---- level n+2 at plane p2 = p-1: from level n+1 planes p-2 (m1), p-1 (c1), p (h1) ----
        const int p2 = p - 1;
        const int sm1 = (it + kRing - 2) % kRing, sc1 = (it + kRing - 1) % kRing;  // ring slots of planes p-2, p-1
        const bool out_pl = it >= 1 && ((p2 >= k0 && p2 < k1) || (robin && p2 == -1));
        const bool own_out = out_pl && warp >= 1 && warp <= kOW;
        float4 c1 = z4, lc1 = z4;
        if (own_out || (out_pl && row_gy)) {
            c1 = ring4(ring_h, sc1, drow);
            lc1 = ring4(ring_l, sc1, drow);
        }
        if (own_out) {
            const float* yh = ring_h + sc1 * T2::ring_slot;
            const float* yl = ring_l + sc1 * T2::ring_slot;
            const float4 m1 = ring4(ring_h, sm1, drow), lm1 = ring4(ring_l, sm1, drow);
            const float4 ys = *reinterpret_cast<const float4*>(yh + drow - kDX2);
            const float4 yn = *reinterpret_cast<const float4*>(yh + drow + kDX2);
            const float4 lys = *reinterpret_cast<const float4*>(yl + drow - kDX2);
            const float4 lyn = *reinterpret_cast<const float4*>(yl + drow + kDX2);
            const float gl = __shfl_up_sync(0xffffffffu, c1.w, 1), gll = __shfl_up_sync(0xffffffffu, lc1.w, 1);
            const float gr = __shfl_down_sync(0xffffffffu, c1.x, 1), grl = __shfl_down_sync(0xffffffffu, lc1.x, 1);
            const bool p2_in = p2 >= 0 && p2 < L.nz;
            if (lane >= 1 && lane <= 30 && row_in && p2_in) {
                float4 ho = z4, lo = z4, dout = z4;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float xl = e == 0 ? gl : el(c1, e - 1), xr = e == 3 ? gr : el(c1, e + 1);
                    const float lxl = e == 0 ? gll : el(lc1, e - 1), lxr = e == 3 ? grl : el(lc1, e + 1);
                    float a, b, c;
                    f32k_update(xl, xr, el(ys, e), el(yn, e), el(m1, e), el(h1, e), el(c1, e), lxl, lxr, el(lys, e),
                                el(lyn, e), el(lm1, e), el(l1, e), el(lc1, e), el(d1c, e), el(sc_, e), nu2, a, b, c);
                    set(ho, e, a);
                    set(lo, e, b);
                    set(dout, e, c);
                }
                const long long q = L.at(xa, j1, p2);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (xc[e] == 0) {
                        hi_n[q + e] = el(ho, e);
                        lo_n[q + e] = lo_encode(el(ho, e), el(lo, e));
                        d_out[q + e] = el(dout, e);
                    }
            }
            // Robin ghosts of level n+2 next to this tile: x faces (the lanes holding x = -1 or nx, rows of the tile),
            // z faces (plane -1 here; plane nz after the march)
            if (robin && row_in && p2_in) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((xc[e] == 1 && xa + e >= x0 - 1) || (xc[e] == 2 && xa + e <= x0 + kOX)) {
                        const bool lo_face = xc[e] == 1;
                        const float gi = lo_face ? (e == 3 ? gr : el(c1, e + 1)) : (e == 0 ? gl : el(c1, e - 1));
                        const float li = lo_face ? (e == 3 ? grl : el(lc1, e + 1)) : (e == 0 ? gll : el(lc1, e - 1));
                        const float2 ab = coef(B, lo_face ? 0 : 1, (long long)p2 * L.ny + j1);
                        float a, b;
                        robin_update_f32k(ab.x, ab.y, el(c1, e), el(lc1, e), gi, li, a, b);
                        const long long q = L.at(xa + e, j1, p2);
                        hi_n[q] = a;
                        lo_n[q] = lo_encode(a, b);
                    }
            }
            if (robin && row_in && p2 == -1 && lane >= 1 && lane <= 30) {
                const long long q = L.at(xa, j1, -1);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (xc[e] == 0) {
                        const float2 ab = coef(B, 4, (long long)j1 * L.nx + xa + e);
                        float a, b;
                        robin_update_f32k(ab.x, ab.y, el(c1, e), el(lc1, e), el(h1, e), el(l1, e), a, b);
                        hi_n[q + e] = a;
                        lo_n[q + e] = lo_encode(a, b);
                    }
            }
        }
        // the y-face ghost rows of level n+2 next to this tile (row -1 in the first row of tiles, row ny in the tile
        // that holds row ny-1), by the warp whose level-(n+1) row is that ghost row
        if (out_pl && row_gy && p2 >= 0 && p2 < L.nz && lane >= 1 && lane <= 30) {
            const float* yh = ring_h + sc1 * T2::ring_slot;
            const float* yl = ring_l + sc1 * T2::ring_slot;
            const int rin = j1 < 0 ? drow + kDX2 : drow - kDX2;  // the interior row next to the ghost row
            const float4 hin = *reinterpret_cast<const float4*>(yh + rin);
            const float4 lin = *reinterpret_cast<const float4*>(yl + rin);
            const long long q = L.at(xa, j1, p2);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (xc[e] == 0) {
                    const float2 ab = coef(B, j1 < 0 ? 2 : 3, (long long)p2 * L.nx + xa + e);
                    float a, b;
                    robin_update_f32k(ab.x, ab.y, el(c1, e), el(lc1, e), el(hin, e), el(lin, e), a, b);
                    hi_n[q + e] = a;
                    lo_n[q + e] = lo_encode(a, b);
                }
        }
        // shift the queues: level n, level n+1, and the increments / source of plane p for the next level n+2
        hm0 = hc0;
        lm0 = lc0;
        hc0 = hp0;
        lc0 = lp0;
        d1c = d1;
        sc_ = s0;
    }
    // copies still in flight (only after a wait gave up) must land before the block ends
    if (threadIdx.x == 0 && !ok)
        for (int i = issued - kS2 > 0 ? issued - kS2 : 0; i < issued; ++i)
            mbar_wait(smem_addr(&bar_full[i % kS2]), (unsigned)((i / kS2) & 1), err);
    // Robin z face at plane nz, by the last chunk: from level n+1 planes nz (c1) and nz-1 (m1), still in the ring
    if (ok && robin && k1 == L.nz && row_in && warp >= 1 && warp <= kOW && lane >= 1 && lane <= 30) {
        const int last = iters - 1;
        const float4 c1 = ring4(ring_h, last % kRing, drow), lc1 = ring4(ring_l, last % kRing, drow);
        const float4 m1 = ring4(ring_h, (last + kRing - 1) % kRing, drow);
        const float4 lm1 = ring4(ring_l, (last + kRing - 1) % kRing, drow);
        const long long q = L.at(xa, j1, L.nz);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (xc[e] == 0) {
                const float2 ab = coef(B, 5, (long long)j1 * L.nx + xa + e);
                float a, b;
                robin_update_f32k(ab.x, ab.y, el(c1, e), el(lc1, e), el(m1, e), el(lm1, e), a, b);
                hi_n[q + e] = a;
                lo_n[q + e] = lo_encode(a, b);
            }
    }
}

constexpr int kZ2 = 32;  // level-(n+2) planes per block

// tensor maps of the staged level-n state with this kernel's boxes: hi[0..1], lo[0..1], dlt[0..1], s
int tma2_maps(hg_grid* g) {
    if (g->tm2_ready) return HG_OK;
    const Layout& L = g->L;
    int rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = tma_encode(&g->tm2[0 + b], g->phi[b], L, 4, kHX2, kHR2))) return rc;
        if ((rc = tma_encode(&g->tm2[2 + b], g->lo[b], L, 2, kLX2, kHR2))) return rc;
        if ((rc = tma_encode(&g->tm2[4 + b], g->dlt[b], L, 4, kDX2, kR1))) return rc;
    }
    if ((rc = tma_encode(&g->tm2[6], g->rho, L, 4, kDX2, kR1))) return rc;
    g->tm2_ready = 1;
    return HG_OK;
}

}  // namespace

// two fused compensated-float sub-steps, cur -> 1 - cur (dlt dcur -> 1 - dcur); Dirichlet and Robin grids
int launch_temporal2_tma(hg_grid* g) {
    if (g->prec != HG_PREC_F32K || !g->dlt[1] || g->bc == HG_BC_PERIODIC)
        return fail(HG_ERR_STATE, "the TMA-staged depth-2 kernel needs a Dirichlet or Robin f32k grid with two dlt buffers");
    int rc = tma2_maps(g);
    if (rc) return rc;
    static unsigned long long attr_done = 0;
    if ((rc = smem_attr_once((const void*)k_temporal2_tma, T2::smem, &attr_done))) return rc;
    const int zb = g->zb > 0 ? (g->zb < g->nz ? g->zb : g->nz) : (g->nz < kZ2 ? g->nz : kZ2);
    SweepArgs A = sweep_args(g, zb);
    A.B.faces = g->bc == HG_BC_ROBIN ? 1 : 0;
    A.B.periodic = 0;
    A.B.xfaces = 0;
    const int c = g->cur;
    dim3 grid((g->nx + kOX - 1) / kOX, (g->ny + kOW - 1) / kOW, (g->nz + zb - 1) / zb);
    if ((rc = prof_begin(g))) return rc;
    k_temporal2_tma<<<grid, 32 * kR1, T2::smem, g->stream>>>(g->tm2[0 + c], g->tm2[2 + c], g->tm2[4 + g->dcur],
                                                                     g->tm2[6], A, (float*)g->dlt[1 - g->dcur],
                                                                     g->derr);
    HG_LAUNCHED("TMA-staged depth-2 sub-step kernel");
    return prof_end(g);
}

}  // namespace hg
