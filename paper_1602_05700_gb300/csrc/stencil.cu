// Single-sweep sub-step of the hyperbolic gravity equation (arXiv 1602.05700, Sec. 1 Eq. HNeq., Sec. 2):
//
//   phi^{n+1} = 2 phi^n - phi^{n-1} + nu^2 sum_{6 nb}(phi^n_nb - phi^n) - s,   s = (c_h dt)^2 4 pi G rho
//
// over the interior of the padded layout.  This file holds the FP64 sweep, the small ghost kernels of a single
// grid's sub-step, the batched launches of many grids, and the host side of a single grid's sub-step; the
// compensated-float sweep itself is the TMA-staged kernel of stencil_tma.cu / sweep_tma.cuh.
//
// * f32k: float storage with compensated increments.  State per cell: hi + lo = phi^n (a float and its
//   rounding remainder, stored as a 16-bit code, cell.cuh) and dlt = phi^n - phi^{n-1}.  The sub-step is
//       dlt' = dlt + (nu^2 (L(hi) + L(lo)) - s),   (hi', lo') = hi + (lo + dlt')  by Fast2Sum,
//   so phi keeps ~36 bits: 24 bytes of HBM traffic per cell (read hi 4, lo 2, dlt 4, s 4; write hi' 4, lo' 2,
//   dlt' 4).  hi/lo ping-pong between two buffers (neighbours are read), dlt is updated in place.
// * f64: double storage, phi^{n+1} written over phi^{n-1}: 32 bytes per cell.  The update's 15 FP64 operations
//   (cell.cuh) run partly in integer instructions with the same bits (lap_int.cuh); GB300's FP64 rate and the
//   integer issue bound the kernel, not HBM.
// The stored "rho" array holds the scaled source s = (c_h dt)^2 4 pi G (rho - rho_bar).
//
// FP64 work mapping: a warp owns one y-row of 128 (or 32) consecutive x cells (4 or 1 per lane, two 16-byte accesses
// or one 8-byte access per lane) and marches in z through a chunk of planes.  The -z / centre / +z planes are a
// register queue; x neighbours come from the adjacent lanes by warp shuffles (the two warp-edge cells load one
// scalar each); y neighbours are the rows of the sibling warps, read through L1.  Ragged tails in x, y and z are
// masked (lanes beyond nx store nothing; the vector reads of the last group stay inside the padded row).
#include "cell.cuh"
#include "hg_internal.cuh"
#include "sweep_f32k.cuh"
#include "sweep_tma.cuh"

namespace hg {

namespace {

__device__ __forceinline__ double2 ld2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
__device__ __forceinline__ double2 ld2rw(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }


// Boundary work rides in the same launch, after each block's z-march (so it adds no registers to the sweep).  Robin:
// a block next to a face updates the face ghosts that border its own cells -- its rows and planes of an x face, its
// x range and planes of a y face, its x range and rows of a z face -- to level n+1, from level-n values only (the
// ghost and its interior neighbour), which no block of the launch writes.  Every face ghost belongs to exactly one
// block.  Dirichlet ghosts are data.  Periodic: see block_periodic_copies.




// The face ghosts owned by this block, handed to upd in batches of up to 4 (padded index of the ghost, of its
// interior neighbour, ghost number), so that the loads of a batch are issued together.
constexpr int kGB = 4;
struct GhostBatch {
    long long qg[kGB], qi[kGB], t[kGB];
    int n;
};

template <class Where, class Upd>
__device__ __forceinline__ void batched(int count, int tid, int nth, Where&& where, Upd&& upd) {
    for (int base = tid; base < count; base += kGB * nth) {
        GhostBatch gb;
        gb.n = 0;
#pragma unroll
        for (int u = 0; u < kGB; ++u) {
            const int t = base + u * nth;
            if (t < count) {
                where(t, gb.qg[u], gb.qi[u], gb.t[u]);
                gb.n = u + 1;
            }
        }
        upd(gb);
    }
}

template <class Upd>
__device__ __forceinline__ void block_face_ghosts(const Layout& L, const Bnd& B, int x0, int j0, int wy, int k0, int k1,
                                                  int bx, int by, int gx, int gy, Upd&& upd, int tw = 128) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int jn = min(wy, L.ny - j0), xn = min(tw, L.nx - x0), kn = k1 - k0;
    if (bx == 0)
        batched(jn * kn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int j = j0 + t % jn, k = k0 + t / jn;
            qg = L.at(-1, j, k), qi = qg + 1, r = B.off[0] + (long long)k * L.ny + j;
        }, upd);
    if (bx == gx - 1)
        batched(jn * kn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int j = j0 + t % jn, k = k0 + t / jn;
            qg = L.at(L.nx, j, k), qi = qg - 1, r = B.off[1] + (long long)k * L.ny + j;
        }, upd);
    if (by == 0)
        batched(xn * kn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int i = x0 + t % xn, k = k0 + t / xn;
            qg = L.at(i, -1, k), qi = qg + L.pitch, r = B.off[2] + (long long)k * L.nx + i;
        }, upd);
    if (by == gy - 1)
        batched(xn * kn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int i = x0 + t % xn, k = k0 + t / xn;
            qg = L.at(i, L.ny, k), qi = qg - L.pitch, r = B.off[3] + (long long)k * L.nx + i;
        }, upd);
    if (k0 == 0)
        batched(xn * jn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int i = x0 + t % xn, j = j0 + t / xn;
            qg = L.at(i, j, -1), qi = qg + L.plane, r = B.off[4] + (long long)j * L.nx + i;
        }, upd);
    if (k1 == L.nz)
        batched(xn * jn, tid, nth, [&](int t, long long& qg, long long& qi, long long& r) {
            const int i = x0 + t % xn, j = j0 + t / xn;
            qg = L.at(i, j, L.nz), qi = qg - L.plane, r = B.off[5] + (long long)j * L.nx + i;
        }, upd);
}

// f64: C = 4 cells per lane (two double2 accesses) or C = 1 (one double); arithmetic in cell.cuh
template <int C>
struct DC {
    double v[C];
};
template <int C>
__device__ __forceinline__ DC<C> ldd(const double* p, bool ro) {
    DC<C> r;
    if constexpr (C == 4) {
        const double2 a = ro ? ld2(p) : ld2rw(p), b = ro ? ld2(p + 2) : ld2rw(p + 2);
        r.v[0] = a.x;
        r.v[1] = a.y;
        r.v[2] = b.x;
        r.v[3] = b.y;
    } else {
        r.v[0] = ro ? __ldg(p) : *p;
    }
    return r;
}

// The FP64 sweep of tile (bx, by) and z chunk bz: a warp owns a row of 32 C cells (C per lane).
template <int WY, int C, bool UNIFORM>
__device__ __forceinline__ void sweep_f64(const SweepArgs& A, int bx, int by, int bz) {
    constexpr int TW = 32 * C;
    const double* __restrict__ phi_c = (const double*)A.hi_c;
    double* __restrict__ phi_pn = (double*)A.hi_n;
    const double* __restrict__ rho = (const double*)A.rho;
    const Layout& L = A.L;
    const Bnd& B = A.B;
    const double nu2 = A.nu2;
    const int zb = A.zb;
    const int lane = threadIdx.x;
    const int j = by * WY + threadIdx.y;
    const int i0 = bx * TW + lane * C;
    const bool active = i0 < L.nx;  // this lane owns cells
    const bool halo = i0 <= L.nx;   // this lane's group holds cells or the +x ghost
    const bool full = i0 + C - 1 < L.nx;
    const int k0 = bz * zb;
    const int k1 = min(L.nz, k0 + zb);
    DC<C> zero;
#pragma unroll
    for (int e = 0; e < C; ++e) zero.v[e] = 0.0;
    if (j < L.ny && (int)threadIdx.y < WY) {  // rows past ny (or extra warps) only join the epilogue
    long long q = L.at(i0, j, k0);
    DC<C> cm = zero, cc = zero;
    if (halo) {
        cm = ldd<C>(phi_c + q - L.plane, true);
        cc = ldd<C>(phi_c + q, true);
    }
    for (int k = k0; k < k1; ++k, q += L.plane) {
        DC<C> cp = zero, ys = zero, yn = zero, pv = zero, r = zero;
        double xl = 0.0, xr = 0.0;
        if (halo) cp = ldd<C>(phi_c + q + L.plane, true);
        if (active) {
            ys = ldd<C>(phi_c + q - L.pitch, true);
            yn = ldd<C>(phi_c + q + L.pitch, true);
            pv = ldd<C>(phi_pn + q, false);
            r = ldd<C>(rho + q, true);
            if (lane == 0) xl = __ldg(phi_c + q - 1);
            if (lane == 31 && i0 + C <= L.nx) xr = __ldg(phi_c + q + C);
        }
        double sl = __shfl_up_sync(0xffffffffu, cc.v[C - 1], 1);
        double sr = __shfl_down_sync(0xffffffffu, cc.v[0], 1);
        if (lane != 0) xl = sl;
        if (lane != 31) xr = sr;
        if (active) {
            DC<C> o;
#pragma unroll
            for (int e = 0; e < C; ++e) {
                double l = e == 0 ? xl : cc.v[e - 1];
                double rr = e == C - 1 ? xr : cc.v[e + 1];
                o.v[e] = f64_update<UNIFORM>(l, rr, ys.v[e], yn.v[e], cm.v[e], cp.v[e], cc.v[e], pv.v[e], r.v[e], nu2);
            }
            if (!idx_ok(q, C, L.elems, B.err)) {
            } else if (C == 4 && full) {
                st2(phi_pn + q, make_double2(o.v[0], o.v[1]));
                st2(phi_pn + q + 2, make_double2(o.v[C > 2 ? 2 : 0], o.v[C > 3 ? 3 : 0]));
            } else {
#pragma unroll
                for (int e = 0; e < C; ++e)
                    if (i0 + e < L.nx) phi_pn[q + e] = o.v[e];
            }
        }
        cm = cc;
        cc = cp;
    }
    }
    if (B.faces)
        block_face_ghosts(L, B, bx * TW, by * WY, WY, k0, k1, bx, by, A.gx, A.gy, [&](const GhostBatch& gb) {
            double a[kGB], rg[kGB], ri[kGB], pg[kGB], pi[kGB];
#pragma unroll
            for (int u = 0; u < kGB; ++u)
                if (u < gb.n) {
                    a[u] = B.robin[3 * gb.t[u]];
                    rg[u] = B.robin[3 * gb.t[u] + 1];
                    ri[u] = B.robin[3 * gb.t[u] + 2];
                    pg[u] = __ldg(phi_c + gb.qg[u]);
                    pi[u] = __ldg(phi_c + gb.qi[u]);
                }
#pragma unroll
            for (int u = 0; u < kGB; ++u)
                if (u < gb.n && idx_ok(gb.qg[u], 1, L.elems, B.err))
                    phi_pn[gb.qg[u]] = robin_update_f64(a[u], rg[u], ri[u], pg[u], pi[u]);
        }, TW);
    if (B.periodic) {
        __syncthreads();
        block_periodic_copies(L, bx * TW, by * WY, WY, k0, k1, bx, by, A.gx, A.gy, block_tid(), block_nth(),
                              [&](long long q, long long d) {
                                  if (idx_ok(d, 1, L.elems, B.err)) phi_pn[d] = phi_pn[q];
                              }, TW);
    }
}

// UNIFORM: the FP64 forms chosen per warp (batched launches) or per lane (the single-grid sweep), cell.cuh
template <int WY, bool UNIFORM>
__device__ __forceinline__ void sweep_f64_any(const SweepArgs& A, int bx, int by, int bz) {
    if (A.cpl == 1)
        sweep_f64<WY, 1, UNIFORM>(A, bx, by, bz);
    else
        sweep_f64<WY, 4, UNIFORM>(A, bx, by, bz);
}

constexpr int kWY = 8;

// ---- boundary kernels of a single-grid sub-step (one thread per face ghost) ----
// ghost t of the face-major enumeration -> padded indices of the ghost, of its interior neighbour, and of the
// interior cell on the opposite face (the periodic source); 32-bit in-face arithmetic
__device__ __forceinline__ void ghost_cells(const Layout& L, const Bnd& B, int t, long long& qg, long long& qi,
                                            long long& qo) {
    int f = 0, base = 0;
#pragma unroll
    for (int u = 1; u < 6; ++u)
        if (t >= (int)B.off[u]) {
            f = u;
            base = (int)B.off[u];
        }
    const int r = t - base;
    const int na = f < 2 ? L.ny : L.nx;
    const int a = r % na, b = r / na;
    switch (f) {
        case 0: qg = L.at(-1, a, b); qi = qg + 1; qo = L.at(L.nx - 1, a, b); break;
        case 1: qg = L.at(L.nx, a, b); qi = qg - 1; qo = L.at(0, a, b); break;
        case 2: qg = L.at(a, -1, b); qi = qg + L.pitch; qo = L.at(a, L.ny - 1, b); break;
        case 3: qg = L.at(a, L.ny, b); qi = qg - L.pitch; qo = L.at(a, 0, b); break;
        case 4: qg = L.at(a, b, -1); qi = qg + L.plane; qo = L.at(a, b, L.nz - 1); break;
        default: qg = L.at(a, b, L.nz); qi = qg - L.plane; qo = L.at(a, b, 0); break;
    }
}

// Robin: ghosts of level n+1 from level n (runs before the sweep; the sweep neither reads nor writes them).  The
// x faces (whose ghosts are strided in memory) are done by the compensated-float sweep itself, so for those grids
// this kernel covers the y and z faces only (t0 = first y-face ghost).
__global__ void __launch_bounds__(256) k_ghosts_robin(const SweepArgs A, int t0) {
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int)A.B.off[6]) return;
    if (((A.B.zskip & 1) && t >= (int)A.B.off[4] && t < (int)A.B.off[5]) || ((A.B.zskip & 2) && t >= (int)A.B.off[5]))
        return;  // a slab interface: the caller supplies that ghost plane
    long long qg, qi, qo;
    ghost_cells(A.L, A.B, t, qg, qi, qo);
    if (A.prec == HG_PREC_F32K) {
        const float* hc = (const float*)A.hi_c;
        const lo_t* lc = (const lo_t*)A.lo_c;
        const float2 ab = A.B.robin32[t];
        const float hg = __ldg(hc + qg), hi = __ldg(hc + qi);
        float gh, gl;
        robin_update_f32k(ab.x, ab.y, hg, lo_decode(hg, lc[qg]), hi, lo_decode(hi, lc[qi]), gh, gl);
        if (!idx_ok(qg, 1, A.L.elems, A.B.err)) return;
        ((float*)A.hi_n)[qg] = gh;
        ((lo_t*)A.lo_n)[qg] = lo_encode(gh, gl);
    } else {
        const double* pc = (const double*)A.hi_c;
        const double* R = A.B.robin;
        if (!idx_ok(qg, 1, A.L.elems, A.B.err)) return;
        ((double*)A.hi_n)[qg] = robin_update_f64(R[3 * t], R[3 * t + 1], R[3 * t + 2], __ldg(pc + qg), __ldg(pc + qi));
    }
}

// periodic: ghosts of level n+1 are copies of the new values on the opposite face (runs after the sweep)
__global__ void __launch_bounds__(256) k_ghosts_periodic(const SweepArgs A, int t0) {
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int)A.B.off[6]) return;
    long long qg, qi, qo;
    ghost_cells(A.L, A.B, t, qg, qi, qo);
    if (A.prec == HG_PREC_F32K) {
        ((float*)A.hi_n)[qg] = ((const float*)A.hi_n)[qo];
        ((lo_t*)A.lo_n)[qg] = ((const lo_t*)A.lo_n)[qo];
    } else {
        ((double*)A.hi_n)[qg] = ((const double*)A.hi_n)[qo];
    }
}

int zchunk(const hg_grid* g) {
    // compensated-float grids (TMA-staged sweep): short chunks, many blocks -- the stage ring hides the z warm-up,
    // and fine blocks balance the SMs (measured at 512^3: 8 planes beat 16-64)
    if (g->prec == HG_PREC_F32K) return g->nz < 8 ? g->nz : 8;
    // enough blocks for several waves on 152 SMs without making the z warm-up (2 planes) a large fraction; Robin
    // grids want about twice as many blocks (the blocks at the x faces also update the face ghosts, and finer
    // blocks balance that extra work better: measured 0.630 against 0.651 ms per sub-step at 512^3)
    long long xy = (long long)((g->nx + 127) / 128) * ((g->ny + kWY - 1) / kWY);
    long long want = 152LL * 8 * (g->bc == HG_BC_ROBIN ? 6 : 3);
    long long nzb = (want + xy - 1) / xy;
    if (nzb < 1) nzb = 1;
    int zb = (int)((g->nz + nzb - 1) / nzb);
    if (zb < 8) zb = 8;
    if (zb > g->nz) zb = g->nz;
    return zb;
}

template <int WY>
__global__ void __launch_bounds__(32 * WY, 2) k_step_f64(const SweepArgs A) {
    sweep_f64_any<WY, false>(A, blockIdx.x, blockIdx.y, blockIdx.z);
}

// entry of block b in a prefix table of n entries
__device__ __forceinline__ int batch_entry(const unsigned* __restrict__ first, int n, unsigned b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One launch for the sub-step of many grids: block b belongs to the entry e with first[e] <= b < first[e+1]
// (binary search in the prefix table).  Compensated-float entries run the TMA-staged sweep (their tensor maps live in
// the table, in global memory; the issuing thread acquires them through the tensormap proxy before its first copy),
// FP64 entries the register-staged FP64 sweep on the first kTmaWY warps, with the last warp joining only its
// boundary epilogue.  Grids of both precisions share the launch, so FP64-bound and HBM-bound blocks run side by side.
template <int WY, int S>
__global__ void __launch_bounds__(32 * (WY + 1), 2) k_step_batch(const TmaEntry* __restrict__ tab,
                                                                 const unsigned* __restrict__ first, int n) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[2 * S];
    const unsigned b = blockIdx.x;
    const int lo = batch_entry(first, n, b);
    const TmaEntry& E = tab[lo];
    const unsigned local = b - __ldg(first + lo);
    const int bx = (int)(local % E.A.gx), by = (int)((local / E.A.gx) % E.A.gy), bz = (int)(local / (E.A.gx * E.A.gy));
    if (E.A.prec == HG_PREC_F32K) {
        if (threadIdx.y == WY && threadIdx.x == 0)  // the producer's issuing thread
            for (int m = 0; m < 4; ++m)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E.m[m]) : "memory");
        tma_sweep<WY, S>(&E.m[0], &E.m[1], &E.m[2], &E.m[3], E.A, bx, by, bz, E.err, smem, bars);
    } else {
        sweep_f64_any<WY, true>(E.A, bx, by, bz);
    }
}

// The two halves of a batched sub-step as launches of their own (the split mode of the batch): compensated-float
// entries only, with the single-grid TMA sweep's launch shape (3 blocks per SM), and FP64 entries only, with the
// single-grid FP64 sweep's (8 warps, 2 blocks per SM).  Each half gets the registers of its own sweep instead of the
// larger of the two.
template <int WY, int S>
__global__ void __launch_bounds__(32 * (WY + 1), 3) k_batch_tma(const TmaEntry* __restrict__ tab,
                                                                const unsigned* __restrict__ first, int n) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[2 * S];
    const int e = batch_entry(first, n, blockIdx.x);
    const TmaEntry& E = tab[e];
    const unsigned local = blockIdx.x - __ldg(first + e);
    const int bx = (int)(local % E.A.gx), by = (int)((local / E.A.gx) % E.A.gy), bz = (int)(local / (E.A.gx * E.A.gy));
    if (threadIdx.y == WY && threadIdx.x == 0)
        for (int m = 0; m < 4; ++m)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&E.m[m]) : "memory");
    tma_sweep<WY, S>(&E.m[0], &E.m[1], &E.m[2], &E.m[3], E.A, bx, by, bz, E.err, smem, bars);
}

template <int WY>
__global__ void __launch_bounds__(32 * WY, 2) k_batch_f64(const TmaEntry* __restrict__ tab,
                                                          const unsigned* __restrict__ first, int n) {
    const int e = batch_entry(first, n, blockIdx.x);
    const SweepArgs& A = tab[e].A;
    const unsigned local = blockIdx.x - __ldg(first + e);
    sweep_f64_any<WY, true>(A, (int)(local % A.gx), (int)((local / A.gx) % A.gy), (int)(local / (A.gx * A.gy)));
}

}  // namespace

// the sweep arguments of grid g for the sub-step cur -> 1 - cur, with z chunks of zb planes (0 = default rule)
int f64_cells_per_lane(int nx) {
    const long long w4 = (nx + 127) / 128 * 128LL, w1 = (nx + 31) / 32 * 32LL;
    return w1 < w4 ? 1 : 4;
}

SweepArgs sweep_args(const hg_grid* g, int zb, int cpl) {
    SweepArgs A;
    const int nxt = 1 - g->cur;
    A.hi_c = g->phi[g->cur];
    A.lo_c = g->lo[g->cur];
    A.hi_n = g->phi[nxt];
    A.lo_n = g->lo[nxt];
    A.dlt = g->dlt[g->dcur];
    A.rho = g->rho;
    A.L = g->L;
    A.nu2 = g->nu2;
    A.nu2f = (float)g->nu2;
    A.zb = zb > 0 ? (zb < g->nz ? zb : g->nz) : zchunk(g);
    A.prec = g->prec;
    A.exact = g->texact;
    A.cpl = g->prec == HG_PREC_F64 ? (cpl > 0 ? cpl : f64_cells_per_lane(g->nx)) : 4;
    A.gx = (g->nx + 32 * A.cpl - 1) / (32 * A.cpl);
    A.gy = (g->ny + kWY - 1) / kWY;
    A.B.faces = g->bc == HG_BC_ROBIN ? 1 : 0;
    A.B.periodic = g->bc == HG_BC_PERIODIC ? 1 : 0;
    A.B.xfaces = 0;
    A.B.zskip = g->ziface;
    A.B.err = g->derr;
    A.B.robin32 = g->robin32;
    A.B.robin = g->robin;
    for (int f = 0; f < 7; ++f) A.B.off[f] = g->F.off[f];
    return A;
}

unsigned sweep_blocks(const SweepArgs& A) { return A.gx * A.gy * (unsigned)((A.L.nz + A.zb - 1) / A.zb); }

// A single grid's sub-step: [Robin ghost kernel] -> sweep -> [periodic ghost kernel].
// Compensated-float grids: the TMA-staged sweep writes all Robin ghosts of level n+1 (x/y faces by its producer
// warp from the staged level-n values, z faces by the first and last chunk) and copies the periodic x-face ghosts;
// the periodic kernel covers the y and z faces with coalesced accesses.  FP64 grids: all ghosts in the small
// kernels.
int launch_step_single(hg_grid* g) {
    SweepArgs A = sweep_args(g, g->zb);
    const int robin = A.B.faces, periodic = A.B.periodic;
    const bool f32k = g->prec == HG_PREC_F32K;
    A.B.faces = 0;
    A.B.periodic = 0;
    if (f32k && periodic) A.B.xfaces = HG_BC_PERIODIC;
    const int t0r = f32k ? (int)A.B.off[6] : 0;  // first ghost left to the Robin kernel (none for f32k)
    const int t0p = f32k ? (int)A.B.off[2] : 0;  // first ghost left to the periodic kernel
    if (robin && t0r < A.B.off[6]) {
        k_ghosts_robin<<<(unsigned)((A.B.off[6] - t0r + 255) / 256), 256, 0, g->stream>>>(A, t0r);
        HG_LAUNCHED("Robin ghost kernel");
    }
    int rc = prof_begin(g);
    if (rc) return rc;
    if (f32k) {
        SweepArgs At = A;
        At.B.faces = robin;  // x/y-face Robin ghosts by the producer warp
        if ((rc = launch_sweep_f32k_tma(g, At))) return rc;
    } else {
        k_step_f64<kWY><<<dim3(A.gx, A.gy, (g->nz + A.zb - 1) / A.zb), dim3(32, kWY), 0, g->stream>>>(A);
        HG_LAUNCHED("stencil sub-step kernel");
    }
    if ((rc = prof_end(g))) return rc;
    if (periodic) {
        k_ghosts_periodic<<<(unsigned)((A.B.off[6] - t0p + 255) / 256), 256, 0, g->stream>>>(A, t0p);
        HG_LAUNCHED("periodic ghost kernel");
    }
    return HG_OK;
}

int launch_batch_class(cudaStream_t st, bool f64, const TmaEntry* tab, const unsigned* first, int n,
                       unsigned total_blocks) {
    if (n < 1 || total_blocks == 0) return HG_OK;
    if (f64) {
        k_batch_f64<kWY><<<total_blocks, dim3(32, kWY), 0, st>>>(tab, first, n);
    } else {
        static unsigned long long attr_done = 0;
        const int smem = kStages * StageGeom<kTmaWY>::bytes;
        int rc = smem_attr_once((const void*)k_batch_tma<kTmaWY, kStages>, smem, &attr_done);
        if (rc) return rc;
        k_batch_tma<kTmaWY, kStages><<<total_blocks, dim3(32, kTmaWY + 1), smem, st>>>(tab, first, n);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, f64 ? "batched FP64 sub-step kernel" : "batched float sub-step kernel");
    return HG_OK;
}

int launch_step_batch(cudaStream_t st, const TmaEntry* tab, const unsigned* first, int n, unsigned total_blocks) {
    static unsigned long long attr_done = 0;
    const int smem = kStages * StageGeom<kTmaWY>::bytes;
    int rc = smem_attr_once((const void*)k_step_batch<kTmaWY, kStages>, smem, &attr_done);
    if (rc) return rc;
    k_step_batch<kTmaWY, kStages><<<total_blocks, dim3(32, kTmaWY + 1), smem, st>>>(tab, first, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batched sub-step kernel");
    return HG_OK;
}

}  // namespace hg
