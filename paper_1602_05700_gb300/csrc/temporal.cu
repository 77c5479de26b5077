// Temporal blocking: K consecutive sub-steps of the hyperbolic gravity equation per round trip through HBM
// (arXiv 1602.05700, Sec. 2: rho is frozen during the wave sub-steps of a hydro step, so K sub-steps can be fused
// without reading the source again).  FP32-compensated state only (hi + lo = phi^n with lo stored as a 16-bit
// code, dlt = phi^n - phi^{n-1}).  The levels computed in registers keep lo as a float, or, in the grid's exact
// mode, round it through its code exactly as a store and a load would (lo_round), so that nothing depends on
// whether a level passed through memory.
//
// A block of 32 x 32 threads owns a 32 x 32 column region of the x-y plane and marches in z through a chunk of
// output planes.  Level 0 (the state at sub-step n) is read once per plane; level t = 1..K is computed one plane
// behind level t-1 (a z pipeline), each level keeping its last three planes (hi, lo) and last two dlt in registers.
// The x/y neighbours of the plane being updated come from a shared-memory copy of level t-1's middle plane
// (double-buffered so one barrier per level suffices).  Level t is valid on the region shrunk by t cells on each
// side, so the 32 - 2K inner columns are written at level K: the K-cell halos are recomputed redundantly by the
// neighbouring blocks instead of being exchanged.  K = 3..8 are built (at K >= 5 the K levels' registers no longer
// fit the 64 a thread of a 1024-thread block gets, and some spill: deep fusion is there for completeness of the
// depth sweep, not for speed).
//
// Boundary cells inside the region follow the boundary condition at every level: Dirichlet ghosts keep their
// data, Robin ghosts take the radiation-condition update (the same float-pair formula as the single-sweep ghost
// kernel),
// periodic regions load wrapped coordinates and are all interior.  Output tiles cover x in [-1, nx], y in [-1, ny]
// and z in [-1, nz], so the face ghosts of level n+K (Robin updates, periodic copies) are written too.  Every update uses the arithmetic of cell.cuh,
// so K fused sub-steps give bit-for-bit the result of K single sweeps.
//
// HBM bytes per cell per K sub-steps: read hi, lo, dlt, rho + write hi, lo, dlt = 24 B (plus halo re-reads, which
// the neighbouring blocks mostly find in L2), i.e. 24/K B per cell-update against 24 B for a single sweep.
#include "cell.cuh"
#include "hg_internal.cuh"

namespace hg {

namespace {

constexpr int TB = 32;  // region side (threads per side)

struct TParams {
    const float* hi_c;
    const lo_t* lo_c;
    const float* d_c;
    const float* rho;  // scaled source s
    float* hi_n;
    lo_t* lo_n;
    float* d_n;
    const float2* robin32;  // (alpha, beta) per face ghost rounded to float, Robin only
    Layout L;
    Faces F;
    float nu2;
    int bc;
    int zchunk;
    int exact;  // inner levels round their compensation through the 16-bit code (bit-identical to single sweeps)
    int* err;   // the grid's device error word (debug index checks)
};

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// One code path for every block.  EDGE = false is used when the block's whole 32 x 32 region lies inside the domain
// in x and y: no per-cell classification at all.  EDGE = true classifies each column once (interior, x-face ghost,
// y-face ghost, or outside) and each plane per level (interior or ghost plane, uniform over the block); ghost cells
// follow their boundary condition, cells outside the domain keep whatever they hold.  No cell tests whether it lies
// in the shrinking valid window: cells near the region edge compute values from unused padding, and those values
// never reach the written inner 32 - 2K columns (each level's valid region shrinks by one cell per side).
template <int K, bool EDGE>
__device__ __forceinline__ void region_sweep(const TParams& P, float2 (*sh)[TB + 2][TB + 2]) {
    constexpr int W = TB - 2 * K;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const Layout& L = P.L;
    const bool periodic = P.bc == HG_BC_PERIODIC;
    const bool robin = P.bc == HG_BC_ROBIN;
    const int x = -1 + (int)blockIdx.x * W + tx - K;
    const int y = -1 + (int)blockIdx.y * W + ty - K;
    const int z0 = -1 + (int)blockIdx.z * P.zchunk;
    const int z1 = min(L.nz + 1, z0 + P.zchunk);  // output planes [z0, z1)

    bool col_int = true, col_fx = false, col_fy = false, loadable = true;
    int xw = x, yw = y;
    if (EDGE) {
        if (periodic) {
            xw = wrap(x, L.nx);
            yw = wrap(y, L.ny);
        } else {
            const bool xin = x >= 0 && x < L.nx, yin = y >= 0 && y < L.ny;
            const bool xg = x == -1 || x == L.nx, yg = y == -1 || y == L.ny;
            col_int = xin && yin;
            col_fx = xg && yin;
            col_fy = xin && yg;
            loadable = x >= -1 && x <= L.nx && y >= -1 && y <= L.ny;
        }
    }
    const bool out_col = tx >= K && tx < TB - K && ty >= K && ty < TB - K && x >= -1 && x <= L.nx && y >= -1 &&
                         y <= L.ny;
    const long long col = loadable ? L.at(xw, yw, 0) : 0;
    const float* hi_c = P.hi_c + col;
    const lo_t* lo_c = P.lo_c + col;
    const float* d_c = P.d_c + col;
    const float* rs = P.rho + col;

    float qh[K][3], ql[K][3], dq[K][2], rq[K + 1];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        qh[t][0] = qh[t][1] = qh[t][2] = 0.f;
        ql[t][0] = ql[t][1] = ql[t][2] = 0.f;
        dq[t][0] = dq[t][1] = 0.f;
    }
#pragma unroll
    for (int t = 0; t <= K; ++t) rq[t] = 0.f;

    // level-0 plane p of this column; pw is p wrapped into [0, nz) for periodic boundaries
    auto load = [&](int p, int pw, float& h, float& l, float& d, float& r) {
        if (!loadable || (!periodic && (p < -1 || p > L.nz))) {
            h = l = d = r = 0.f;
            return;
        }
        const long long o = (long long)(periodic ? pw : p) * L.plane;
        h = __ldg(hi_c + o);
        l = lo_decode(h, lo_c[o]);
        d = __ldg(d_c + o);
        r = __ldg(rs + o);
    };

    int pw = periodic ? wrap(z0 - K, L.nz) : 0;
    float nh, nl, nd, nr;
    load(z0 - K, pw, nh, nl, nd, nr);
    int par = 0;  // parity of the shared-memory buffer for level 1 of this plane
    for (int p = z0 - K; p < z1 + K; ++p) {
        const float h0 = nh, l0 = nl, d0 = nd, r0 = nr;
        if (periodic && ++pw == L.nz) pw = 0;
        if (p + 1 < z1 + K) load(p + 1, pw, nh, nl, nd, nr);
        qh[0][0] = qh[0][1];
        qh[0][1] = qh[0][2];
        qh[0][2] = h0;
        ql[0][0] = ql[0][1];
        ql[0][1] = ql[0][2];
        ql[0][2] = l0;
        dq[0][0] = dq[0][1];
        dq[0][1] = d0;
#pragma unroll
        for (int t = K; t > 0; --t) rq[t] = rq[t - 1];
        rq[0] = r0;
#pragma unroll
        for (int t = 1; t <= K; ++t) {
            const int pt = p - t;  // plane level t computes in this iteration
            const float c = qh[t - 1][1], lc = ql[t - 1][1];
            const float dprev = dq[t - 1][0];
            const int b = par ^ ((t - 1) & 1);  // consecutive levels alternate buffers, also across planes
            sh[b][ty + 1][tx + 1] = make_float2(c, lc);
            __syncthreads();
            float oh = c, ol = lc, od = dprev;
            const bool zin = periodic || (pt >= 0 && pt < L.nz);
            const bool zg = !periodic && (pt == -1 || pt == L.nz);
            if (col_int && zin) {
                const float2 xl = sh[b][ty + 1][tx], xr = sh[b][ty + 1][tx + 2];
                const float2 ys = sh[b][ty][tx + 1], yn = sh[b][ty + 2][tx + 1];
                f32k_update(xl.x, xr.x, ys.x, yn.x, qh[t - 1][0], qh[t - 1][2], c, xl.y, xr.y, ys.y, yn.y,
                            ql[t - 1][0], ql[t - 1][2], lc, dprev, rq[t], P.nu2, oh, ol, od);
                if (t < K && P.exact) ol = lo_round(oh, ol);
            } else if (robin && ((col_int && zg) || (EDGE && (col_fx || col_fy) && zin))) {
                float2 in;
                long long row;
                if (EDGE && col_fx) {
                    in = x < 0 ? sh[b][ty + 1][tx + 2] : sh[b][ty + 1][tx];
                    row = P.F.off[x < 0 ? 0 : 1] + (long long)pt * L.ny + y;
                } else if (EDGE && col_fy) {
                    in = y < 0 ? sh[b][ty + 2][tx + 1] : sh[b][ty][tx + 1];
                    row = P.F.off[y < 0 ? 2 : 3] + (long long)pt * L.nx + x;
                } else {
                    in = pt < 0 ? make_float2(qh[t - 1][2], ql[t - 1][2]) : make_float2(qh[t - 1][0], ql[t - 1][0]);
                    row = P.F.off[pt < 0 ? 4 : 5] + (long long)y * L.nx + x;
                }
                const float2 ab = P.robin32[row];
                robin_update_f32k(ab.x, ab.y, c, lc, in.x, in.y, oh, ol);
                if (t < K && P.exact) ol = lo_round(oh, ol);
            }
            if (t < K) {
                qh[t][0] = qh[t][1];
                qh[t][1] = qh[t][2];
                qh[t][2] = oh;
                ql[t][0] = ql[t][1];
                ql[t][1] = ql[t][2];
                ql[t][2] = ol;
                dq[t][0] = dq[t][1];
                dq[t][1] = od;
            } else if (out_col && pt >= z0 && pt < z1) {
                const long long q = L.at(x, y, pt);
                if (!idx_ok(q, 1, L.elems, P.err)) {
                } else if (periodic) {
                    // interior cells, and the face ghosts as copies of the wrapped cells (the same values the
                    // blocks owning those cells compute, from the same inputs)
                    const int nout = (x < 0 || x >= L.nx) + (y < 0 || y >= L.ny) + (pt < 0 || pt >= L.nz);
                    if (nout <= 1 && pt >= -1 && pt <= L.nz) {
                        P.hi_n[q] = oh;
                        P.lo_n[q] = lo_encode(oh, ol);
                        if (nout == 0) P.d_n[q] = od;
                    }
                } else if (col_int && zin) {
                    P.hi_n[q] = oh;
                    P.lo_n[q] = lo_encode(oh, ol);
                    P.d_n[q] = od;
                } else if (robin && ((col_int && zg) || (EDGE && (col_fx || col_fy) && zin))) {
                    P.hi_n[q] = oh;
                    P.lo_n[q] = lo_encode(oh, ol);
                }
            }
        }
        if (K & 1) par ^= 1;
    }
}

template <int K>
__global__ void __launch_bounds__(TB* TB, 1) k_temporal_f32k(const TParams P) {
    constexpr int W = TB - 2 * K;
    __shared__ float2 sh[2][TB + 2][TB + 2];  // padded by one cell: edge threads read (unused) padding
    const int xr0 = -1 + (int)blockIdx.x * W - K, yr0 = -1 + (int)blockIdx.y * W - K;
    const bool inside = xr0 >= 0 && xr0 + TB <= P.L.nx && yr0 >= 0 && yr0 + TB <= P.L.ny;
    if (inside)
        region_sweep<K, false>(P, sh);
    else
        region_sweep<K, true>(P, sh);
}

template <int K>
int launch_k(hg_grid* g, const TParams& P, int zchunk) {
    constexpr int W = TB - 2 * K;
    dim3 block(TB, TB);
    dim3 grid((g->nx + 2 + W - 1) / W, (g->ny + 2 + W - 1) / W, (g->nz + 2 + zchunk - 1) / zchunk);
    k_temporal_f32k<K><<<grid, block, 0, g->stream>>>(P);
    HG_LAUNCHED("temporal sub-step kernel");
    return HG_OK;
}

}  // namespace

int launch_temporal(hg_grid* g, int k) {
    if (g->prec != HG_PREC_F32K || !g->dlt[1]) return fail(HG_ERR_STATE, "temporal blocking needs an f32k grid");
    if (k == 2 && g->bc != HG_BC_PERIODIC) return launch_temporal2_tma(g);  // the TMA-staged depth-2 kernel
    int nxt = 1 - g->cur;
    TParams P;
    P.hi_c = (const float*)g->phi[g->cur];
    P.lo_c = (const lo_t*)g->lo[g->cur];
    P.d_c = (const float*)g->dlt[g->dcur];
    P.rho = (const float*)g->rho;
    P.hi_n = (float*)g->phi[nxt];
    P.lo_n = (lo_t*)g->lo[nxt];
    P.d_n = (float*)g->dlt[1 - g->dcur];
    P.robin32 = g->robin32;
    P.L = g->L;
    P.F = g->F;
    P.nu2 = (float)g->nu2;
    P.bc = g->bc;
    int zchunk = 64;
    if (zchunk > g->nz + 2) zchunk = g->nz + 2;
    P.zchunk = zchunk;
    P.exact = g->texact;
    P.err = g->derr;
    int rc = prof_begin(g);
    if (rc) return rc;
    switch (k) {
        case 2: rc = launch_k<2>(g, P, zchunk); break;
        case 3: rc = launch_k<3>(g, P, zchunk); break;
        case 4: rc = launch_k<4>(g, P, zchunk); break;
        case 5: rc = launch_k<5>(g, P, zchunk); break;
        case 6: rc = launch_k<6>(g, P, zchunk); break;
        case 7: rc = launch_k<7>(g, P, zchunk); break;
        case 8: rc = launch_k<8>(g, P, zchunk); break;
        default: return fail(HG_ERR_ARG, "temporal depth %d not built", k);
    }
    if (rc) return rc;
    return prof_end(g);
}

}  // namespace hg
