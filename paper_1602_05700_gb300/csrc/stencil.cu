// Single-sweep sub-step of the hyperbolic gravity equation (arXiv 1602.05700, Sec. 1 Eq. HNeq., Sec. 2):
//
//   phi^{n+1} = 2 phi^n - phi^{n-1} + nu^2 sum_{6 nb}(phi^n_nb - phi^n) - s,   s = (c_h dt)^2 4 pi G rho
//
// over the interior of the padded layout (ghosts are filled by boundary.cu).  One kernel per precision:
//
// * f32k: float storage with compensated increments.  State per cell: hi + lo = phi^n (a float and its
//   rounding remainder) and dlt = phi^n - phi^{n-1}.  The sub-step is
//       dlt' = dlt + (nu^2 (L(hi) + L(lo)) - s),   (hi', lo') = hi + (lo + dlt')  by Fast2Sum,
//   so phi keeps ~48 bits while every array is float: 28 bytes of HBM traffic per cell (read hi, lo, dlt, rho;
//   write hi', lo', dlt').  hi/lo ping-pong between two buffers (neighbours are read), dlt is updated in place.
// * f64: double storage, phi^{n+1} written over phi^{n-1}: 32 bytes per cell.  GB300 issues few FP64
//   instructions per clock (~0.5 T/s), and the update takes 15 of them (cell.cuh), so this kernel is bound by the
//   FP64 pipe, not by HBM.
// The stored "rho" array holds the scaled source s = (c_h dt)^2 4 pi G (rho - rho_bar).
//
// Work mapping (both kernels): a warp owns one y-row of 128 consecutive x cells (4 per lane, one 16-byte access
// per lane for float, two for double) and marches in z through a chunk of planes.  The -z / centre / +z planes
// are a register queue; x neighbours come from the adjacent lanes by warp shuffles (the two warp-edge cells
// load one scalar each); y neighbours are the rows of the sibling warps, read through L1.  Ragged tails in x, y
// and z are masked (lanes beyond nx store nothing; the vector reads of the last group stay inside the padded row).
#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4rw(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ double2 ld2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
__device__ __forceinline__ double2 ld2rw(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

__device__ __forceinline__ float el(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ void set(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

// Robin boundary work rides in the same launch: when `faces` is set, the first z-slice of blocks (scheduled first,
// so it overlaps the sweep) updates every face ghost to level n+1 from level-n values only (the ghost and its
// interior neighbour), which no other block of the launch writes.  The sweep blocks themselves carry no boundary
// code, so the interior path keeps its registers and its memory pipeline.  Dirichlet ghosts are data; periodic
// copies of the new level are made by a small kernel after the sweep (boundary.cu).
struct Bnd {
    int faces;              // 1: Robin ghost blocks present (blockIdx.z == 0)
    const float2* robin32;  // (alpha, beta) per face ghost, compensated float grids
    const double* robin;    // (alpha, beta, gamma) per face ghost, FP64 grids
    long long off[7];       // face offsets in the ghost enumeration (hg::Faces)
};

// face ghost t -> padded indices of the ghost and of its interior neighbour (32-bit in-face arithmetic)
__device__ __forceinline__ void face_pair(const Layout& L, const Bnd& B, long long t, long long& qg, long long& qi) {
    // face index and offset by comparisons (no dynamic indexing of the parameter array, which would go to local
    // memory)
    long long base = 0;
    int f = 0;
#pragma unroll
    for (int u = 1; u < 6; ++u)
        if (t >= B.off[u]) {
            f = u;
            base = B.off[u];
        }
    const int r = (int)(t - base);
    const int na = f < 2 ? L.ny : L.nx;
    const int a = r % na, b = r / na;
    switch (f) {
        case 0: qg = L.at(-1, a, b); qi = qg + 1; break;
        case 1: qg = L.at(L.nx, a, b); qi = qg - 1; break;
        case 2: qg = L.at(a, -1, b); qi = qg + L.pitch; break;
        case 3: qg = L.at(a, L.ny, b); qi = qg - L.pitch; break;
        case 4: qg = L.at(a, b, -1); qi = qg + L.plane; break;
        default: qg = L.at(a, b, L.nz); qi = qg - L.plane; break;
    }
}

__device__ __forceinline__ long long face_thread(long long& stride) {
    stride = (long long)gridDim.x * gridDim.y * blockDim.x * blockDim.y;
    return ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) + threadIdx.y * blockDim.x +
           threadIdx.x;
}

template <int WY>
__global__ void __launch_bounds__(32 * WY) k_step_f32k(const float* __restrict__ hi_c, const float* __restrict__ lo_c,
                                                       float* __restrict__ hi_n, float* __restrict__ lo_n,
                                                       float* __restrict__ dlt, const float* __restrict__ rho, Layout L,
                                                       float nu2, int zb, Bnd B) {
    if (B.faces && blockIdx.z == 0) {  // Robin ghosts of level n+1
        long long stride;
        for (long long t = face_thread(stride); t < B.off[6]; t += stride) {
            long long qg, qi;
            face_pair(L, B, t, qg, qi);
            const float2 ab = B.robin32[t];
            float gh, gl;
            robin_update_f32k(ab.x, ab.y, __ldg(hi_c + qg), __ldg(lo_c + qg), __ldg(hi_c + qi), __ldg(lo_c + qi), gh, gl);
            hi_n[qg] = gh;
            lo_n[qg] = gl;
        }
        return;
    }
    const int lane = threadIdx.x;
    const int j = blockIdx.y * WY + threadIdx.y;
    if (j >= L.ny) return;  // whole warp
    const int i0 = blockIdx.x * 128 + lane * 4;
    const bool active = i0 < L.nx;  // this lane owns cells
    const bool halo = i0 <= L.nx;   // this lane's group holds cells or the +x ghost (read for its left neighbour)
    const bool full = i0 + 3 < L.nx;
    const int k0 = (blockIdx.z - B.faces) * zb;
    const int k1 = min(L.nz, k0 + zb);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    long long q = L.at(i0, j, k0);
    float4 hm = z4, hc = z4, lm = z4, lc = z4;
    if (halo) {
        hm = ld4(hi_c + q - L.plane);
        lm = ld4(lo_c + q - L.plane);
        hc = ld4(hi_c + q);
        lc = ld4(lo_c + q);
    }
    for (int k = k0; k < k1; ++k, q += L.plane) {
        float4 hp = z4, lp = z4, hs = z4, hn = z4, ls = z4, ln = z4, d = z4, r = z4;
        float hl = 0.f, hr = 0.f, ll = 0.f, lr = 0.f;
        if (halo) {
            hp = ld4(hi_c + q + L.plane);
            lp = ld4(lo_c + q + L.plane);
        }
        if (active) {
            hs = ld4(hi_c + q - L.pitch);
            hn = ld4(hi_c + q + L.pitch);
            ls = ld4(lo_c + q - L.pitch);
            ln = ld4(lo_c + q + L.pitch);
            d = ld4rw(dlt + q);
            r = ld4(rho + q);
            if (lane == 0) {
                hl = __ldg(hi_c + q - 1);
                ll = __ldg(lo_c + q - 1);
            }
            if (lane == 31 && i0 + 4 <= L.nx) {
                hr = __ldg(hi_c + q + 4);
                lr = __ldg(lo_c + q + 4);
            }
        }
        float shl = __shfl_up_sync(0xffffffffu, hc.w, 1), sll = __shfl_up_sync(0xffffffffu, lc.w, 1);
        float shr = __shfl_down_sync(0xffffffffu, hc.x, 1), slr = __shfl_down_sync(0xffffffffu, lc.x, 1);
        if (lane != 0) {
            hl = shl;
            ll = sll;
        }
        if (lane != 31) {
            hr = shr;
            lr = slr;
        }
        if (active) {
            float4 ho, lo, dout;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float xl = e == 0 ? hl : el(hc, e - 1);
                float xr = e == 3 ? hr : el(hc, e + 1);
                float lxl = e == 0 ? ll : el(lc, e - 1);
                float lxr = e == 3 ? lr : el(lc, e + 1);
                float a, b, c;
                f32k_update(xl, xr, el(hs, e), el(hn, e), el(hm, e), el(hp, e), el(hc, e), lxl, lxr, el(ls, e),
                            el(ln, e), el(lm, e), el(lp, e), el(lc, e), el(d, e), el(r, e), nu2, a, b, c);
                set(ho, e, a);
                set(lo, e, b);
                set(dout, e, c);
            }
            if (full) {
                st4(hi_n + q, ho);
                st4(lo_n + q, lo);
                st4(dlt + q, dout);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < L.nx) {
                        hi_n[q + e] = el(ho, e);
                        lo_n[q + e] = el(lo, e);
                        dlt[q + e] = el(dout, e);
                    }
            }
        }
        hm = hc;
        hc = hp;
        lm = lc;
        lc = lp;
    }
}

// f64: 4 cells per lane as two double2 (arithmetic in cell.cuh)
struct D4 {
    double v[4];
};
__device__ __forceinline__ D4 ldd4(const double* p) {
    double2 a = ld2(p), b = ld2(p + 2);
    D4 r;
    r.v[0] = a.x;
    r.v[1] = a.y;
    r.v[2] = b.x;
    r.v[3] = b.y;
    return r;
}
__device__ __forceinline__ D4 ldd4rw(const double* p) {
    double2 a = ld2rw(p), b = ld2rw(p + 2);
    D4 r;
    r.v[0] = a.x;
    r.v[1] = a.y;
    r.v[2] = b.x;
    r.v[3] = b.y;
    return r;
}

template <int WY>
__global__ void __launch_bounds__(32 * WY, 3) k_step_f64(const double* __restrict__ phi_c, double* __restrict__ phi_pn,
                                                      const double* __restrict__ rho, Layout L, double nu2, int zb,
                                                      Bnd B) {
    if (B.faces && blockIdx.z == 0) {  // Robin ghosts of level n+1
        long long stride;
        for (long long t = face_thread(stride); t < B.off[6]; t += stride) {
            long long qg, qi;
            face_pair(L, B, t, qg, qi);
            phi_pn[qg] = robin_update(B.robin[3 * t], B.robin[3 * t + 1], __ldg(phi_c + qg), __ldg(phi_c + qi));
        }
        return;
    }
    const int lane = threadIdx.x;
    const int j = blockIdx.y * WY + threadIdx.y;
    if (j >= L.ny) return;
    const int i0 = blockIdx.x * 128 + lane * 4;
    const bool active = i0 < L.nx;  // this lane owns cells
    const bool halo = i0 <= L.nx;   // this lane's group holds cells or the +x ghost
    const bool full = i0 + 3 < L.nx;
    const int k0 = (blockIdx.z - B.faces) * zb;
    const int k1 = min(L.nz, k0 + zb);
    D4 zero;
#pragma unroll
    for (int e = 0; e < 4; ++e) zero.v[e] = 0.0;
    long long q = L.at(i0, j, k0);
    D4 cm = zero, cc = zero;
    if (halo) {
        cm = ldd4(phi_c + q - L.plane);
        cc = ldd4(phi_c + q);
    }
    for (int k = k0; k < k1; ++k, q += L.plane) {
        D4 cp = zero, ys = zero, yn = zero, pv = zero, r = zero;
        double xl = 0.0, xr = 0.0;
        if (halo) cp = ldd4(phi_c + q + L.plane);
        if (active) {
            ys = ldd4(phi_c + q - L.pitch);
            yn = ldd4(phi_c + q + L.pitch);
            pv = ldd4rw(phi_pn + q);
            r = ldd4(rho + q);
            if (lane == 0) xl = __ldg(phi_c + q - 1);
            if (lane == 31 && i0 + 4 <= L.nx) xr = __ldg(phi_c + q + 4);
        }
        double sl = __shfl_up_sync(0xffffffffu, cc.v[3], 1);
        double sr = __shfl_down_sync(0xffffffffu, cc.v[0], 1);
        if (lane != 0) xl = sl;
        if (lane != 31) xr = sr;
        if (active) {
            D4 o;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                double l = e == 0 ? xl : cc.v[e - 1];
                double rr = e == 3 ? xr : cc.v[e + 1];
                o.v[e] = f64_update(l, rr, ys.v[e], yn.v[e], cm.v[e], cp.v[e], cc.v[e], pv.v[e], r.v[e], nu2);
            }
            if (full) {
                st2(phi_pn + q, make_double2(o.v[0], o.v[1]));
                st2(phi_pn + q + 2, make_double2(o.v[2], o.v[3]));
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < L.nx) phi_pn[q + e] = o.v[e];
            }
        }
        cm = cc;
        cc = cp;
    }
}

constexpr int kWY = 8;

int zchunk(const hg_grid* g) {
    // enough blocks for several waves on 152 SMs without making the z warm-up (2 planes) a large fraction
    long long xy = (long long)((g->nx + 127) / 128) * ((g->ny + kWY - 1) / kWY);
    long long want = 152LL * 8 * 3;
    long long nzb = (want + xy - 1) / xy;
    if (nzb < 1) nzb = 1;
    int zb = (int)((g->nz + nzb - 1) / nzb);
    if (zb < 8) zb = 8;
    if (zb > g->nz) zb = g->nz;
    return zb;
}

}  // namespace

int launch_step_single(hg_grid* g) {
    const Layout& L = g->L;
    int zb = zchunk(g);
    dim3 block(32, kWY);
    Bnd B;
    B.faces = g->bc == HG_BC_ROBIN ? 1 : 0;
    B.robin32 = g->robin32;
    B.robin = g->robin;
    for (int f = 0; f < 7; ++f) B.off[f] = g->F.off[f];
    dim3 grid((g->nx + 127) / 128, (g->ny + kWY - 1) / kWY, (g->nz + zb - 1) / zb + B.faces);
    int nxt = 1 - g->cur;
    int rc = prof_begin(g);
    if (rc) return rc;
    if (g->prec == HG_PREC_F32K) {
        k_step_f32k<kWY><<<grid, block, 0, g->stream>>>(
            (const float*)g->phi[g->cur], (const float*)g->lo[g->cur], (float*)g->phi[nxt], (float*)g->lo[nxt],
            (float*)g->dlt[g->dcur], (const float*)g->rho, L, (float)g->nu2, zb, B);
    } else {
        k_step_f64<kWY><<<grid, block, 0, g->stream>>>((const double*)g->phi[g->cur], (double*)g->phi[nxt],
                                                       (const double*)g->rho, L, g->nu2, zb, B);
    }
    HG_LAUNCHED("stencil sub-step kernel");
    return prof_end(g);
}

}  // namespace hg
