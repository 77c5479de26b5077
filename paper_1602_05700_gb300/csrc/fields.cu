// Field movement between the caller's dense arrays and the padded device layout, the gravitational acceleration
// -grad phi (arXiv 1602.05700: the force the hydro step consumes, Sec. 2), and the FP64 diagnostics of Sec. 4
// (Eq. error) and of the steady state (Eq. Poissoneq.).  Reductions are deterministic: fixed grid, per-block
// partial sums, one finishing block.
#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

static_assert(sizeof(lo_t) == sizeof(lo_code), "the compensation code is 16 bits wide");

namespace {

constexpr int kThreads = 256;
constexpr int kPackBlocks = 1216;  // 8 per SM; one partial sum each (fits the reduction scratch)

__device__ __forceinline__ double ld(const void* p, int dtype, long long i) {
    return dtype == HG_DT_F64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}
__device__ __forceinline__ void st(void* p, int dtype, long long i, double v) {
    if (dtype == HG_DT_F64)
        ((double*)p)[i] = v;
    else
        ((float*)p)[i] = (float)v;
}

// value of phi^n at padded index q, in double (F32K: float plus its decoded compensation)
__device__ __forceinline__ double phi_at(int prec, const void* p, const void* lo, long long q) {
    if (prec == HG_PREC_F64) return ((const double*)p)[q];
    return join_f32(((const float*)p)[q], ((const lo_t*)lo)[q]);
}

// visit every interior cell: blocks stride over the rows (j, k), threads over x (coalesced, no per-cell division)
template <class F>
__device__ __forceinline__ void for_cells(const Layout& L, F&& f) {
    const long long rows = (long long)L.ny * L.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % L.ny), k = (int)(row / L.ny);
        const long long base = row * L.nx;
        for (int i = threadIdx.x; i < L.nx; i += blockDim.x) f(i, j, k, base + i);
    }
}

// Source preparation: dst = scale * (src - shift) in the grid's layout and element type, where scale =
// (c dt)^2 4 pi G and shift = mean(rho) for periodic boundaries (else 0).  Float input to a float grid is scaled in
// float (one rounding more than FP64, 6e-8 relative, and no slow FP64 instructions); every other combination in
// FP64.  With SUM the same pass also accumulates sum(src) for the FP64 mass: each thread in compensated float
// (TwoSum) or double, blocks in double, written as one partial per block (deterministic order).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

template <typename TS, typename TD, bool SUM>
__global__ void __launch_bounds__(kThreads) k_pack(const TS* __restrict__ src, TD* __restrict__ dst, Layout L,
                                                   const double* __restrict__ sum, double count, double scale,
                                                   double* partial) {
    float fs = 0.f, fc = 0.f;  // compensated float accumulator (float input)
    double ds = 0.0;           // double accumulator (double input)
    const double shift = sum ? *sum / count : 0.0;  // rho_bar = sum(rho) / cells, read on the device (no host sync)
    const float scale32 = (float)scale, shift32 = (float)shift;
    if constexpr (sizeof(TS) == 4 && sizeof(TD) == 4) {
        if ((L.nx & 3) == 0 && ((uintptr_t)src & 15) == 0) {  // 16-byte groups on both sides
            // a block takes rpb rows at a time (all its threads busy when a row has fewer groups than threads)
            const long long rows = (long long)L.ny * L.nz;
            const int gpr = L.nx >> 2, rpb = gpr >= (int)blockDim.x ? 1 : (int)blockDim.x / gpr;
            const int sub = rpb == 1 ? 0 : (int)threadIdx.x / gpr, i0 = rpb == 1 ? (int)threadIdx.x : (int)threadIdx.x % gpr;
            const int istep = rpb == 1 ? (int)blockDim.x : gpr;
            for (long long row = (long long)blockIdx.x * rpb + sub; row < rows; row += (long long)gridDim.x * rpb) {
                if (sub >= rpb) break;  // threads beyond rpb * gpr
                const int j = (int)(row % L.ny), k = (int)(row / L.ny);
                const float4* s4 = reinterpret_cast<const float4*>(src + row * L.nx);
                float4* d4 = reinterpret_cast<float4*>(dst + L.at(0, j, k));
                for (int i = i0; i < gpr; i += istep) {
                    const float4 x = __ldg(s4 + i);
                    d4[i] = make_float4(scale32 * (x.x - shift32), scale32 * (x.y - shift32), scale32 * (x.z - shift32),
                                        scale32 * (x.w - shift32));
                    if constexpr (SUM) {
                        two_sum_acc(fs, fc, x.x);
                        two_sum_acc(fs, fc, x.y);
                        two_sum_acc(fs, fc, x.z);
                        two_sum_acc(fs, fc, x.w);
                    }
                }
            }
        } else {
            for_cells(L, [&](int i, int j, int k, long long c) {
                const float x = src[c];
                dst[L.at(i, j, k)] = scale32 * (x - shift32);
                if constexpr (SUM) two_sum_acc(fs, fc, x);
            });
        }
    } else {
        for_cells(L, [&](int i, int j, int k, long long c) {
            const TS x = src[c];
            dst[L.at(i, j, k)] = (TD)(scale * ((double)x - shift));
            if constexpr (SUM) {
                if constexpr (sizeof(TS) == 4)
                    two_sum_acc(fs, fc, x);
                else
                    ds += x;
            }
        });
    }
    if constexpr (SUM) {
        __shared__ double sh[32];
        const double v = block_sum(sizeof(TS) == 4 ? (double)fs + (double)fc : ds, sh);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_unpack(int prec, const void* p, const void* lo, void* dst, int ddt, Layout L) {
    for_cells(L, [&](int i, int j, int k, long long c) { st(dst, ddt, c, phi_at(prec, p, lo, L.at(i, j, k))); });
}

__global__ void k_unpack_ghosted(int prec, const void* p, const void* lo, double* dst, Layout L) {
    const int gx = L.nx + 2, gy = L.ny + 2, gz = L.nz + 2;
    const long long rows = (long long)gy * gz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % gy) - 1, k = (int)(row / gy) - 1;
        for (int ii = threadIdx.x; ii < gx; ii += blockDim.x) {
            const int i = ii - 1;
            const int out = (i < 0 || i >= L.nx) + (j < 0 || j >= L.ny) + (k < 0 || k >= L.nz);
            dst[row * gx + ii] = out > 1 ? 0.0 : phi_at(prec, p, lo, L.at(i, j, k));
        }
    }
}

// seed: level n from phi, level n-1 from prev (F64 into the two buffers; F32K: hi/lo split of phi and
// dlt = phi - prev rounded once)
__global__ void k_seed(int prec, const void* phi, const void* prev, int sdt, void* p_cur, void* l_cur, void* p_oth,
                       void* l_oth, void* dlt, Layout L) {
    for_cells(L, [&](int i, int j, int k, long long c) {
        const long long q = L.at(i, j, k);
        const double a = ld(phi, sdt, c);
        const double b = prev ? ld(prev, sdt, c) : a;
        if (prec == HG_PREC_F64) {
            ((double*)p_cur)[q] = a;
            ((double*)p_oth)[q] = b;
        } else {
            float ha, hb;
            lo_t la, lb;
            split_f32(a, ha, la);
            split_f32(b, hb, lb);
            ((float*)p_cur)[q] = ha;
            ((lo_t*)l_cur)[q] = la;
            ((float*)p_oth)[q] = hb;
            ((lo_t*)l_oth)[q] = lb;
            ((float*)dlt)[q] = (float)(a - b);
        }
    });
}

// a = -grad phi by central differences.  Compensated float grids with float output stay in float arithmetic
// ((hi+ - hi-) + (lo+ - lo-)); every other combination evaluates phi = hi + lo (or the double) in FP64.
__global__ void k_accel(int prec, const void* p, const void* lo, void* ax, void* ay, void* az, int ddt, Layout L,
                        double inv2h) {
    for_cells(L, [&](int i, int j, int k, long long c) {
        const long long q = L.at(i, j, k);
        if (prec == HG_PREC_F32K && ddt == HG_DT_F32) {
            const float* h = (const float*)p;
            const lo_t* lc = (const lo_t*)lo;
            auto l = [&](long long u) { return lo_decode(h[u], lc[u]); };
            const float s = (float)inv2h;
            ((float*)ax)[c] = -((h[q + 1] - h[q - 1]) + (l(q + 1) - l(q - 1))) * s;
            ((float*)ay)[c] = -((h[q + L.pitch] - h[q - L.pitch]) + (l(q + L.pitch) - l(q - L.pitch))) * s;
            ((float*)az)[c] = -((h[q + L.plane] - h[q - L.plane]) + (l(q + L.plane) - l(q - L.plane))) * s;
        } else {
            st(ax, ddt, c, -(phi_at(prec, p, lo, q + 1) - phi_at(prec, p, lo, q - 1)) * inv2h);
            st(ay, ddt, c, -(phi_at(prec, p, lo, q + L.pitch) - phi_at(prec, p, lo, q - L.pitch)) * inv2h);
            st(az, ddt, c, -(phi_at(prec, p, lo, q + L.plane) - phi_at(prec, p, lo, q - L.plane)) * inv2h);
        }
    });
}

// Vectorised -grad phi for compensated float grids with float output (the per-hydro-step call): the work mapping
// of the sub-step kernel (a warp per 128-cell x-row, float4 per lane, x neighbours by shuffles, a z register queue)
// and the same arithmetic as k_accel.  HBM bytes per cell: read hi 4, lo 2; write ax, ay, az 12 = 18 B.  The kernel
// waits on its loads (no data reuse hides them), so four blocks per SM (64 registers) beat three (71 registers):
// 0.432 against 0.458 ms at 512^3.
constexpr int kAccWY = 8;
__global__ void __launch_bounds__(32 * kAccWY, 4) k_accel_f32k(const float* __restrict__ hi, const lo_t* __restrict__ lo,
                                                            float* __restrict__ ax, float* __restrict__ ay,
                                                            float* __restrict__ az, Layout L, float s, int zb) {
    const int lane = threadIdx.x;
    const int j = blockIdx.y * kAccWY + threadIdx.y;
    if (j >= L.ny) return;
    const int i0 = blockIdx.x * 128 + lane * 4;
    const bool active = i0 < L.nx, halo = i0 <= L.nx;
    const bool vec = (L.nx & 3) == 0 && i0 + 3 < L.nx;
    const int k0 = blockIdx.z * zb, k1 = min(L.nz, k0 + zb);
    auto ld4 = [](const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); };
    auto ldl4 = [](const lo_t* p) { return __ldg(reinterpret_cast<const uint2*>(p)); };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    long long q = L.at(i0, j, k0);
    float4 hm = z4, hc = z4, lm = z4, lc = z4;
    if (halo) {
        hm = ld4(hi + q - L.plane);
        lm = lo_decode4(hm, ldl4(lo + q - L.plane));
        hc = ld4(hi + q);
        lc = lo_decode4(hc, ldl4(lo + q));
    }
    for (int k = k0; k < k1; ++k, q += L.plane) {
        float4 hp = z4, lp = z4, hs = z4, hn = z4, ls = z4, ln = z4;
        float hl = 0.f, hr = 0.f, ll = 0.f, lr = 0.f;
        if (halo) {
            hp = ld4(hi + q + L.plane);
            lp = lo_decode4(hp, ldl4(lo + q + L.plane));
        }
        if (active) {
            hs = ld4(hi + q - L.pitch);
            hn = ld4(hi + q + L.pitch);
            ls = lo_decode4(hs, ldl4(lo + q - L.pitch));
            ln = lo_decode4(hn, ldl4(lo + q + L.pitch));
            if (lane == 0) {
                hl = __ldg(hi + q - 1);
                ll = lo_decode(hl, lo[q - 1]);
            }
            if (lane == 31 && i0 + 4 <= L.nx) {
                hr = __ldg(hi + q + 4);
                lr = lo_decode(hr, lo[q + 4]);
            }
        }
        const float shl = __shfl_up_sync(0xffffffffu, hc.w, 1), sll = __shfl_up_sync(0xffffffffu, lc.w, 1);
        const float shr = __shfl_down_sync(0xffffffffu, hc.x, 1), slr = __shfl_down_sync(0xffffffffu, lc.x, 1);
        if (lane != 0) {
            hl = shl;
            ll = sll;
        }
        if (lane != 31) {
            hr = shr;
            lr = slr;
        }
        if (active) {
            const float xh[6] = {hl, hc.x, hc.y, hc.z, hc.w, hr}, xl[6] = {ll, lc.x, lc.y, lc.z, lc.w, lr};
            const float hs_[4] = {hs.x, hs.y, hs.z, hs.w}, hn_[4] = {hn.x, hn.y, hn.z, hn.w};
            const float ls_[4] = {ls.x, ls.y, ls.z, ls.w}, ln_[4] = {ln.x, ln.y, ln.z, ln.w};
            const float hm_[4] = {hm.x, hm.y, hm.z, hm.w}, hp_[4] = {hp.x, hp.y, hp.z, hp.w};
            const float lm_[4] = {lm.x, lm.y, lm.z, lm.w}, lp_[4] = {lp.x, lp.y, lp.z, lp.w};
            float ox[4], oy[4], oz[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ox[e] = -((xh[e + 2] - xh[e]) + (xl[e + 2] - xl[e])) * s;
                oy[e] = -((hn_[e] - hs_[e]) + (ln_[e] - ls_[e])) * s;
                oz[e] = -((hp_[e] - hm_[e]) + (lp_[e] - lm_[e])) * s;
            }
            const long long c = ((long long)k * L.ny + j) * L.nx + i0;
            if (vec) {
                *reinterpret_cast<float4*>(ax + c) = make_float4(ox[0], ox[1], ox[2], ox[3]);
                *reinterpret_cast<float4*>(ay + c) = make_float4(oy[0], oy[1], oy[2], oy[3]);
                *reinterpret_cast<float4*>(az + c) = make_float4(oz[0], oz[1], oz[2], oz[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < L.nx) {
                        ax[c + e] = ox[e];
                        ay[c + e] = oy[e];
                        az[c + e] = oz[e];
                    }
            }
        }
        hm = hc;
        hc = hp;
        lm = lc;
        lc = lp;
    }
}

// partial[b*NS + s] for the stats: 0 sum res^2, 1 max|res|, 2 sum (phi - phi_prev)^2, 3 sum phi^2, 4 max|phi|,
// 5 count of non-finite values
constexpr int NS = 6;
constexpr unsigned kStatsMax = (1u << 1) | (1u << 4);

__global__ void __launch_bounds__(kThreads) k_stats(int prec, const void* p, const void* lo, const void* pprev,
                                                    const void* dlt, const void* rho, Layout L, double ih2,
                                                    double inv_cdt2, double* partial) {
    __shared__ double sh[32];
    double a[NS] = {0, 0, 0, 0, 0, 0};
    for_cells(L, [&](int i, int j, int k, long long) {
        const long long q = L.at(i, j, k);
        const double pc = phi_at(prec, p, lo, q);
        double lap = 0.0;
        lap += phi_at(prec, p, lo, q - 1) - pc;
        lap += phi_at(prec, p, lo, q + 1) - pc;
        lap += phi_at(prec, p, lo, q - L.pitch) - pc;
        lap += phi_at(prec, p, lo, q + L.pitch) - pc;
        lap += phi_at(prec, p, lo, q - L.plane) - pc;
        lap += phi_at(prec, p, lo, q + L.plane) - pc;
        double r, d;
        if (prec == HG_PREC_F64) {
            r = ((const double*)rho)[q];
            d = pc - ((const double*)pprev)[q];
        } else {
            r = (double)((const float*)rho)[q];
            d = (double)((const float*)dlt)[q];
        }
        const double res = lap * ih2 - r * inv_cdt2;  // r = s = (c dt)^2 4 pi G (rho - rho_bar)
        a[0] += res * res;
        a[1] = fmax(a[1], fabs(res));
        a[2] += d * d;
        a[3] += pc * pc;
        a[4] = fmax(a[4], fabs(pc));
        if (!isfinite(pc) || !isfinite(d) || !isfinite(r)) a[5] += 1.0;
    });
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double v = block_reduce(a[s], sh, (kStatsMax >> s) & 1u);
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * NS + s] = v;
    }
}

// partial for compare: 0 sum (phi-P)^2, 1 sum P^2, 2 max|phi-P|, 3 max|P|, 4 sum ((phi-P)/P)^2
constexpr int NC = 5;
constexpr unsigned kCmpMax = (1u << 2) | (1u << 3);

__global__ void __launch_bounds__(kThreads) k_compare(int prec, const void* p, const void* lo, const double* P,
                                                      Layout L, double* partial) {
    __shared__ double sh[32];
    double a[NC] = {0, 0, 0, 0, 0};
    for_cells(L, [&](int i, int j, int k, long long c) {
        const double v = phi_at(prec, p, lo, L.at(i, j, k));
        const double b = P[c];
        const double d = v - b;
        a[0] += d * d;
        a[1] += b * b;
        a[2] = fmax(a[2], fabs(d));
        a[3] = fmax(a[3], fabs(b));
        a[4] += (d / b) * (d / b);
    });
#pragma unroll
    for (int s = 0; s < NC; ++s) {
        double v = block_reduce(a[s], sh, (kCmpMax >> s) & 1u);
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * NC + s] = v;
    }
}

__global__ void __launch_bounds__(kThreads) k_sum(const void* src, int dt, long long n, double* partial) {
    __shared__ double sh[32];
    double a = 0.0;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (dt == HG_DT_F32) {
        const float* p = (const float*)src;
        float fs = 0.f, fc = 0.f;  // TwoSum-compensated float accumulation, then double
        const long long n4 = ((uintptr_t)p & 15) == 0 ? n >> 2 : 0;
        for (long long c = tid; c < n4; c += nt) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(p) + c);
            two_sum_acc(fs, fc, x.x);
            two_sum_acc(fs, fc, x.y);
            two_sum_acc(fs, fc, x.z);
            two_sum_acc(fs, fc, x.w);
        }
        for (long long c = 4 * n4 + tid; c < n; c += nt) two_sum_acc(fs, fc, p[c]);
        a = (double)fs + (double)fc;
    } else {
        const double* p = (const double*)src;
        for (long long c = tid; c < n; c += nt) a += p[c];
    }
    double v = block_sum(a, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// finish: out[s] = sum (or max, per bit of maxmask) over blocks of partial[b*ns + s], fixed order
__global__ void __launch_bounds__(kThreads) k_finish_mixed(const double* partial, int nblocks, int ns,
                                                           unsigned maxmask, double* out) {
    __shared__ double sh[32];
    for (int s = 0; s < ns; ++s) {
        const bool is_max = (maxmask >> s) & 1u;
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            double x = partial[(long long)b * ns + s];
            v = is_max ? fmax(v, x) : v + x;
        }
        v = block_reduce(v, sh, is_max);
        if (threadIdx.x == 0) out[s] = v;
    }
}

// one block per row up to a cap (rows are strided by the grid)
inline unsigned cells_blocks(const hg_grid* g) {
    long long rows = (long long)(g->ny + 2) * (g->nz + 2);
    return (unsigned)(rows < 152 * 64 ? rows : 152 * 64);
}

}  // namespace

template <bool SUM>
static int launch_pack(hg_grid* g, const void* src, int dtype, const double* sum, double scale) {
    const unsigned blocks = SUM ? (unsigned)kPackBlocks : cells_blocks(g);
    const double count = (double)g->nx * g->ny * g->nz;
    if (dtype == HG_DT_F32 && g->prec == HG_PREC_F32K)
        k_pack<float, float, SUM><<<blocks, kThreads, 0, g->stream>>>((const float*)src, (float*)g->rho, g->L, sum,
                                                                      count, scale, g->red);
    else if (dtype == HG_DT_F32)
        k_pack<float, double, SUM><<<blocks, kThreads, 0, g->stream>>>((const float*)src, (double*)g->rho, g->L, sum,
                                                                       count, scale, g->red);
    else if (g->prec == HG_PREC_F32K)
        k_pack<double, float, SUM><<<blocks, kThreads, 0, g->stream>>>((const double*)src, (float*)g->rho, g->L, sum,
                                                                       count, scale, g->red);
    else
        k_pack<double, double, SUM><<<blocks, kThreads, 0, g->stream>>>((const double*)src, (double*)g->rho, g->L,
                                                                        sum, count, scale, g->red);
    HG_LAUNCHED("source preparation kernel");
    return HG_OK;
}

// Store the scaled source s = (c dt)^2 4 pi G (rho - rho_bar) and leave sum(rho) (FP64-accurate) in g->dsum on the
// device; nothing here waits for the GPU.  Periodic boundaries need the mean before scaling: a sum pass, then the
// pack reading the sum from device memory; otherwise one fused pass.
int prepare_source(hg_grid* g, const void* src, int dtype) {
    int rc;
    g->mass_pending = 1;
    if (g->bc == HG_BC_PERIODIC) {
        if ((rc = reduce_sum(g, src, dtype, g->dsum))) return rc;
        return launch_pack<false>(g, src, dtype, g->dsum, g->src);
    }
    if ((rc = launch_pack<true>(g, src, dtype, nullptr, g->src))) return rc;
    k_finish_mixed<<<1, kThreads, 0, g->stream>>>(g->red, kPackBlocks, 1, 0u, g->dsum);
    HG_LAUNCHED("sum finish kernel");
    return HG_OK;
}

// Bring the mass and mean density of the last hg_set_density to the host (waits for the stream once per density)
int sync_mass(hg_grid* g) {
    if (!g->mass_pending) return HG_OK;
    double sum = 0.0;
    HG_CUDA(cudaMemcpyAsync(&sum, g->dsum, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    g->mass = sum * g->h * g->h * g->h;
    g->rho_bar = g->bc == HG_BC_PERIODIC ? sum / ((double)g->nx * g->ny * g->nz) : 0.0;
    g->mass_pending = 0;
    return HG_OK;
}

int unpack_phi(hg_grid* g, void* dst, int dtype) {
    k_unpack<<<cells_blocks(g), kThreads, 0, g->stream>>>(g->prec, g->phi[g->cur], g->lo[g->cur], dst, dtype, g->L);
    HG_LAUNCHED("unpack kernel");
    return HG_OK;
}

int unpack_phi_ghosted(hg_grid* g, double* dst) {
    k_unpack_ghosted<<<cells_blocks(g), kThreads, 0, g->stream>>>(g->prec, g->phi[g->cur], g->lo[g->cur], dst, g->L);
    HG_LAUNCHED("ghosted unpack kernel");
    return HG_OK;
}

int set_phi_device(hg_grid* g, const void* phi, const void* prev, int dtype) {
    int oth = 1 - g->cur;
    k_seed<<<cells_blocks(g), kThreads, 0, g->stream>>>(g->prec, phi, prev, dtype, g->phi[g->cur], g->lo[g->cur],
                                                        g->phi[oth], g->lo[oth], g->dlt[g->dcur], g->L);
    HG_LAUNCHED("seed kernel");
    return HG_OK;
}

int accel(hg_grid* g, void* ax, void* ay, void* az, int dtype) {
    const bool aligned = ((uintptr_t)ax | (uintptr_t)ay | (uintptr_t)az) % 16 == 0;
    if (g->prec == HG_PREC_F32K && dtype == HG_DT_F32 && aligned) {
        const int zb = g->nz < 8 ? g->nz : 8;  // short z chunks: more blocks in flight (measured 0.459 ms at 512^3
                                                // against 0.489 ms with 32-plane chunks)
        dim3 block(32, kAccWY), grid((g->nx + 127) / 128, (g->ny + kAccWY - 1) / kAccWY, (g->nz + zb - 1) / zb);
        k_accel_f32k<<<grid, block, 0, g->stream>>>((const float*)g->phi[g->cur], (const lo_t*)g->lo[g->cur],
                                                    (float*)ax, (float*)ay, (float*)az, g->L,
                                                    (float)(1.0 / (2.0 * g->h)), zb);
    } else {
        k_accel<<<cells_blocks(g), kThreads, 0, g->stream>>>(g->prec, g->phi[g->cur], g->lo[g->cur], ax, ay, az,
                                                             dtype, g->L, 1.0 / (2.0 * g->h));
    }
    HG_LAUNCHED("acceleration kernel");
    return HG_OK;
}

int stats(hg_grid* g, hg_stats* s) {
    int rc = sync_mass(g);
    if (rc) return rc;
    if ((rc = device_error(g))) return rc;
    k_stats<<<kRedBlocks, kThreads, 0, g->stream>>>(g->prec, g->phi[g->cur], g->lo[g->cur], g->phi[1 - g->cur],
                                                    g->dlt[g->dcur], g->rho, g->L, 1.0 / (g->h * g->h),
                                                    1.0 / ((g->c * g->dt) * (g->c * g->dt)), g->red);
    HG_LAUNCHED("stats kernel");
    k_finish_mixed<<<1, kThreads, 0, g->stream>>>(g->red, kRedBlocks, NS, kStatsMax, g->dres);
    HG_LAUNCHED("stats finish kernel");
    double r[NS];
    HG_CUDA(cudaMemcpyAsync(r, g->dres, sizeof r, cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    const double n = (double)g->nx * g->ny * g->nz;
    s->mass = g->mass;
    s->residual_rms = sqrt(r[0] / n);
    s->residual_max = r[1];
    s->change_rel = r[3] > 0.0 ? sqrt(r[2] / r[3]) : 0.0;
    s->phi_max = r[4];
    s->step = g->step;
    s->nonfinite = r[5] > 0.0 ? 1 : 0;
    return HG_OK;
}

int compare(hg_grid* g, const double* P, double out[3]) {
    k_compare<<<kRedBlocks, kThreads, 0, g->stream>>>(g->prec, g->phi[g->cur], g->lo[g->cur], P, g->L, g->red);
    HG_LAUNCHED("compare kernel");
    k_finish_mixed<<<1, kThreads, 0, g->stream>>>(g->red, kRedBlocks, NC, kCmpMax, g->dres);
    HG_LAUNCHED("compare finish kernel");
    double r[NC];
    HG_CUDA(cudaMemcpyAsync(r, g->dres, sizeof r, cudaMemcpyDeviceToHost, g->stream));
    HG_CUDA(cudaStreamSynchronize(g->stream));
    const double n = (double)g->nx * g->ny * g->nz;
    out[0] = sqrt(r[0] / r[1]);
    out[1] = r[2] / r[3];
    out[2] = sqrt(r[4] / n);
    return HG_OK;
}

int reduce_sum(hg_grid* g, const void* dense, int dtype, double* out_dev) {
    long long n = (long long)g->nx * g->ny * g->nz;
    k_sum<<<kPackBlocks, kThreads, 0, g->stream>>>(dense, dtype, n, g->red);
    HG_LAUNCHED("sum kernel");
    k_finish_mixed<<<1, kThreads, 0, g->stream>>>(g->red, kPackBlocks, 1, 0u, out_dev);
    HG_LAUNCHED("sum finish kernel");
    return HG_OK;
}

}  // namespace hg
