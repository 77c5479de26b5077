// Two fused sub-steps per HBM round trip (temporal blocking, depth 2) of the compensated-float sub-step, staged by
// TMA (arXiv 1602.05700, Sec. 2: rho is frozen during the wave sub-steps of a hydro step, so consecutive sub-steps
// can be fused without reading the source again).  Dirichlet and Robin grids; periodic grids use temporal.cu.
//
// A block writes a tile of 128 x-cells x 8 rows of level n+2 over a chunk of z planes, marching in z.  Level n+1 is
// needed on the tile grown by one cell: rows j0-1 .. j0+8 (r = 0 .. 9) over cells x0-1 .. x0+128.
//   * warp w (w = 1 .. 8) computes level n+1 of its row w over the 128 cells of the tile (4 cells per lane),
//     writes it into a two-slot shared ring, then level n+2 of the same row one plane behind; warp 0 computes
//     level n+1 of the two halo rows 0 and 9;
//   * the helper warp (warp 9) issues the bulk-tensor copies of level n (plane by plane into a ring of 4 stages:
//     hi and lo-code rows j0-2 .. j0+9, dlt and s rows j0-1 .. j0+8, all over cells x0-4 .. x0+131), computes
//     level n+1 of the two halo columns x0-1 and x0+128 (20 single cells: no halo is recomputed by whole warps,
//     so a 512-cell row takes exactly 4 tiles) and writes the level-(n+2) x-face ghosts.
// In z the two levels form a pipeline: iteration `it` computes level n+1 at plane p = k0-1+it (own row's -z/centre
// planes of level n in registers, +z and the y rows from the stages) and level n+2 at plane p-1 (own row's level
// n+1 planes p-2, p-1, p in registers, the neighbouring rows and halo columns at p-1 from the ring); one block
// barrier ends each iteration, after which the helper refills the stage of plane p with plane p+4.
//
// Face ghosts follow the boundary condition exactly as a single sweep writes them (Dirichlet: the data, unchanged;
// Robin: the radiation update from the ghost and its interior neighbour), and the level-(n+2) face ghosts bordering
// the tile are written with the new level.  Level n+1 never passes through memory, so its compensations stay floats
// (slightly more accurate than the 16-bit code a stored level keeps); with the grid's exact mode set
// (hg_set_temporal_exact) they go through the code as a store and a load would (lo_round4) and every cell update is
// the single sweep's scalar form (cell.cuh), so the result is then bit-identical to two single sweeps; the default
// mode runs the update on packed float pairs.
//
// HBM bytes per cell for the two sub-steps: 24 (read hi, lo, dlt, s; write hi, lo, dlt) plus the halo rows and
// planes of neighbouring tiles (mostly served by L2).  Every wait is bounded in time; a wait that gives up sets the
// grid's error word and makes the whole block skip its remaining work (all warps still meet every barrier).
#include "sweep_tma.cuh"

namespace hg {

namespace {

constexpr int kFX = 128;              // level-(n+2) cells of a tile row
constexpr int kFY = 8;                // level-(n+2) rows of a tile
constexpr int kFR = kFY + 2;          // level-(n+1) rows (one warp each): y = j0-1+r, r = 0 .. 9
constexpr int kFH = kFY + 4;          // staged level-n hi / lo rows: y = j0-2 .. j0+9 (stage row = r + 1)
constexpr int kFC = kFX + 8;          // staged columns: x = x0-4 .. x0+131 (column = x - x0 + 4)
constexpr int kFS = 4;                // stage ring depth
constexpr int kFHelper = kFY + 1;     // warp index of the helper (warps 0 .. 8 own the rows)
constexpr int kFThreads = 32 * (kFY + 2);

struct F2 {
    static constexpr int h_tx = kFH * kFC * 4;
    static constexpr int l_tx = kFH * kFC * 2;
    static constexpr int d_tx = kFR * kFC * 4;
    static constexpr int h_off = 0;
    static constexpr int l_off = align128(h_tx);
    static constexpr int d_off = l_off + align128(l_tx);
    static constexpr int s_off = d_off + align128(d_tx);
    static constexpr int stage = s_off + align128(d_tx);
    static constexpr int ring_off = kFS * stage;
    static constexpr int ring_slot = kFR * kFC;  // floats per slot (hi; the lo slots follow all hi slots)
    static constexpr int smem = ring_off + 2 * 2 * ring_slot * 4;
};

__device__ __forceinline__ float2 coef(const Bnd& B, int f, long long t) { return B.robin32[B.off[f] + t]; }

// Robin update of four ghosts (face f, coefficient indices t0 .. t0+3) from the ghost values (hg, lg) and their
// interior neighbours (hin, lin); only the first `n` (1..4) of them exist (a ragged tile's last group)
__device__ __forceinline__ void robin4(const Bnd& B, int f, long long t0, const float4& hg, const float4& lg,
                                       const float4& hin, const float4& lin, float4& ho, float4& lo, int n = 4) {
    ho = hg;
    lo = lg;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (e >= n) break;
        const float2 ab = coef(B, f, t0 + e);
        float a, b;
        robin_update_f32k(ab.x, ab.y, el(hg, e), el(lg, e), el(hin, e), el(lin, e), a, b);
        set(ho, e, a);
        set(lo, e, b);
    }
}

// One block: RAGGED is set for the last tile in x when nx is not a multiple of 128 (then the +x ghost lies inside
// the tile and every lane classifies its cells); otherwise the x halo columns are the helper's.
template <bool RAGGED, bool EXACT>
__device__ __forceinline__ void fused2_block(const CUtensorMap* m_hi, const CUtensorMap* m_lo, const CUtensorMap* m_d,
                                             const CUtensorMap* m_s, const SweepArgs& A, float* __restrict__ d_out,
                                             int* err, unsigned char* smem, unsigned long long* bar_full,
                                             volatile int* abort_flag) {
    const Layout& L = A.L;
    const Bnd& B = A.B;
    const bool robin = B.faces != 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kFX, j0 = blockIdx.y * kFY;
    const int k0 = blockIdx.z * A.zb, k1 = min(L.nz, k0 + A.zb);
    const int nload = k1 - k0 + 3;  // level-n planes k0-1 .. k1+1: stage index i holds plane k0-1+i
    const int iters = k1 - k0 + 2;  // level n+1 at planes k0-1 .. k1
    const float nu2 = A.nu2f;
    float* ring_h = (float*)(smem + F2::ring_off);
    float* ring_l = ring_h + 2 * F2::ring_slot;
    float* __restrict__ hi_n = (float*)A.hi_n;
    lo_t* __restrict__ lo_n = (lo_t*)A.lo_n;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    auto stage_ptr = [&](int i) { return smem + (i % kFS) * F2::stage; };
    auto issue = [&](int i) {  // level-n plane k0-1+i (padded plane k0+i) into stage i % kFS
        const uint32_t full = smem_addr(&bar_full[i % kFS]);
        unsigned char* st = stage_ptr(i);
        mbar_expect_tx(full, F2::h_tx + F2::l_tx + 2 * F2::d_tx);
        tma_load_3d(smem_addr(st + F2::h_off), m_hi, x0, j0 - 1, k0 + i, full);
        tma_load_3d(smem_addr(st + F2::l_off), m_lo, x0, j0 - 1, k0 + i, full);
        tma_load_3d(smem_addr(st + F2::d_off), m_d, x0, j0, k0 + i, full);
        tma_load_3d(smem_addr(st + F2::s_off), m_s, x0, j0, k0 + i, full);
    };
    // wait for stage i; gives up (and tells the block) after the bound
    auto wait_stage = [&](int i) -> bool {
        if (*abort_flag) return false;
        if (mbar_wait(smem_addr(&bar_full[i % kFS]), (unsigned)((i / kFS) & 1), err)) return true;
        *abort_flag = 1;
        return false;
    };
    auto Hs = [&](int i) { return (const float*)(stage_ptr(i) + F2::h_off); };
    auto Ls = [&](int i) { return (const lo_t*)(stage_ptr(i) + F2::l_off); };
    auto Ds = [&](int i) { return (const float*)(stage_ptr(i) + F2::d_off); };
    auto Ss = [&](int i) { return (const float*)(stage_ptr(i) + F2::s_off); };
    auto rh = [&](int slot, int r, int col) { return ring_h + slot * F2::ring_slot + r * kFC + col; };
    auto rl = [&](int slot, int r, int col) { return ring_l + slot * F2::ring_slot + r * kFC + col; };

    if (warp == kFHelper) {
        // ---------------- helper: copies, level n+1 of the halo columns, level-(n+2) x-face ghosts ----------------
        int issued = 0;
        if (lane == 0)
            for (; issued < kFS && issued < nload; ++issued) issue(issued);
        // lanes 0..9: column x0-1 of row r = lane; lanes 16..25: column x0+128 of row r = lane-16
        const int side = lane >> 4, r = lane & 15;
        const int col = side ? kFX + 4 : 3, xh = side ? x0 + kFX : x0 - 1;
        const int y = j0 - 1 + r;
        const bool mine = r < kFR && y >= 0 && y < L.ny && (side ? (!RAGGED && xh <= L.nx) : true);
        const bool ghost = mine && (xh == -1 || xh == L.nx);  // an x-face ghost (only the tiles at the faces)
        const int sr = r + 1;
        float hm = 0.f, lm = 0.f;  // level n at plane p-1 of this lane's cell
        for (int it = 0; it < iters; ++it) {
            const int p = k0 - 1 + it;
            bool ok = it > 0 || wait_stage(0);
            ok = ok && wait_stage(it + 1);
            ok = __all_sync(0xffffffffu, ok);
            if (ok && mine) {
                const float* H = Hs(it);
                const lo_t* Lo = Ls(it);
                const float hc = H[sr * kFC + col], lc = lo_decode(hc, Lo[sr * kFC + col]);
                if (p >= k0 && p < k1) {  // the ring needs the halo columns at the tile's own planes only
                    float a = hc, b = lc;
                    if (ghost) {
                        if (robin) {
                            const int ci = side ? col - 1 : col + 1;  // the interior neighbour
                            const float hin = H[sr * kFC + ci];
                            const float2 ab = coef(B, side, (long long)p * L.ny + y);
                            robin_update_f32k(ab.x, ab.y, hc, lc, hin, lo_decode(hin, Lo[sr * kFC + ci]), a, b);
                            if (EXACT) b = lo_round(a, b);
                        }
                    } else {
                        const float* Hp = Hs(it + 1);
                        const lo_t* Lp = Ls(it + 1);
                        const float xl = H[sr * kFC + col - 1], xr = H[sr * kFC + col + 1];
                        const float ys = H[(sr - 1) * kFC + col], yn = H[(sr + 1) * kFC + col];
                        const float zp = Hp[sr * kFC + col];
                        float c;
                        f32k_update(xl, xr, ys, yn, hm, zp, hc, lo_decode(xl, Lo[sr * kFC + col - 1]),
                                    lo_decode(xr, Lo[sr * kFC + col + 1]), lo_decode(ys, Lo[(sr - 1) * kFC + col]),
                                    lo_decode(yn, Lo[(sr + 1) * kFC + col]), lm, lo_decode(zp, Lp[sr * kFC + col]), lc,
                                    Ds(it)[r * kFC + col], Ss(it)[r * kFC + col], nu2, a, b, c);
                        if (EXACT) b = lo_round(a, b);
                    }
                    *rh(it & 1, r, col) = a;
                    *rl(it & 1, r, col) = b;
                }
                hm = hc;
                lm = lc;
            }
            // level-(n+2) x-face ghosts at plane q = p-1 (Robin), rows 1..8, from the ring written last iteration
            const int q = p - 1;
            if (ok && ghost && robin && r >= 1 && r <= kFY && q >= k0 && q < k1) {
                const int slot = (it - 1) & 1, ci = side ? col - 1 : col + 1;
                const float2 ab = coef(B, side, (long long)q * L.ny + y);
                float a, b;
                robin_update_f32k(ab.x, ab.y, *rh(slot, r, col), *rl(slot, r, col), *rh(slot, r, ci),
                                  *rl(slot, r, ci), a, b);
                const long long qi = L.at(xh, y, q);
                if (idx_ok(qi, 1, L.elems, B.err)) {
                    hi_n[qi] = a;
                    lo_n[qi] = lo_encode(a, b);
                }
            }
            __syncthreads();
            if (lane == 0 && !*abort_flag && it + kFS < nload) {  // every warp is done with plane p's stage
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(it + kFS);
                issued = it + kFS + 1;
            }
        }
        // copies still in flight (only after a wait gave up) must land before the block ends
        if (lane == 0 && *abort_flag)
            for (int i = issued - kFS > 0 ? issued - kFS : 0; i < issued; ++i)
                mbar_wait(smem_addr(&bar_full[i % kFS]), (unsigned)((i / kFS) & 1), err);
        return;
    }

    // ---------------- row warps ------------------------------------------------------------------------------------
    // warp w = 1..8: level n+1 of row w and level n+2 of the same row one plane behind; warp 0: level n+1 of the two
    // halo rows 0 and 9 (y = j0-1 and j0+8), and the level-(n+2) y-face ghost row when one of them is a ghost row
    const int xa = x0 + 4 * lane;  // first cell of this lane's group
    const int col = 4 + 4 * lane;  // its stage / ring column
    // RAGGED tiles: the class of each of the lane's cells in x -- 0 interior, 2 the +x ghost, 3 beyond it
    int xc[4] = {0, 0, 0, 0};
    if (RAGGED)
#pragma unroll
        for (int e = 0; e < 4; ++e) xc[e] = xa + e < L.nx ? 0 : xa + e == L.nx ? 2 : 3;
    const int nlive = RAGGED ? max(0, min(4, L.nx - xa)) : 4;  // interior cells of the group

    struct Row {
        int r, y, sr;
        bool in, ghost, live, out;
    };
    auto make_row = [&](int r) {
        Row R;
        R.r = r;
        R.y = j0 - 1 + r;
        R.sr = r + 1;
        R.in = R.y >= 0 && R.y < L.ny;                // an interior row
        R.ghost = R.y == -1 || R.y == L.ny;           // a y-face ghost row
        R.live = R.in || R.ghost;
        R.out = r >= 1 && r <= kFY;                   // has level n+2 in this tile
        return R;
    };
    // level n+1 of row R at plane p (iteration it) from level n (z window hm0/lm0 = plane p-1, hc0/lc0 = plane p,
    // loaded here), written into ring slot it & 1; h1, l1, d1: the new level, s0: the source at p
    auto level1 = [&](const Row& R, int it, float4& hm0, float4& lm0, float4& hc0, float4& lc0, float4& h1,
                      float4& l1, float4& d1, float4& s0) {
        const int p = k0 - 1 + it, r = R.r, sr = R.sr, y = R.y;
        const float* H = Hs(it);
        const lo_t* Lo = Ls(it);
        const float4 d0 = lds4(Ds(it) + r * kFC + col);
        s0 = lds4(Ss(it) + r * kFC + col);
        h1 = hc0;  // ghosts without an update (Dirichlet data) keep level n
        l1 = lc0;
        d1 = d0;
        if (R.in && p >= 0 && p < L.nz) {
            // interior plane of an interior row: the stencil (RAGGED: the +x ghost cell by its boundary rule)
            const float* Hp = Hs(it + 1);
            const float4 hp0 = lds4(Hp + sr * kFC + col);
            const float4 lp0 = lo_decode4(hp0, ldsl4(Ls(it + 1) + sr * kFC + col));
            const float4 hs = lds4(H + (sr - 1) * kFC + col), hn = lds4(H + (sr + 1) * kFC + col);
            const float4 ls = lo_decode4(hs, ldsl4(Lo + (sr - 1) * kFC + col));
            const float4 ln = lo_decode4(hn, ldsl4(Lo + (sr + 1) * kFC + col));
            float hl = __shfl_up_sync(0xffffffffu, hc0.w, 1), ll = __shfl_up_sync(0xffffffffu, lc0.w, 1);
            float hr = __shfl_down_sync(0xffffffffu, hc0.x, 1), lr = __shfl_down_sync(0xffffffffu, lc0.x, 1);
            if (lane == 0) {
                hl = H[sr * kFC + 3];
                ll = lo_decode(hl, Lo[sr * kFC + 3]);
            }
            if (lane == 31) {
                hr = H[sr * kFC + kFX + 4];
                lr = lo_decode(hr, Lo[sr * kFC + kFX + 4]);
            }
            if (EXACT)
                f32k_update4_scalar(hc0, lc0, hl, ll, hr, lr, hs, hn, hm0, hp0, ls, ln, lm0, lp0, d0, s0, nu2, h1, l1, d1);
            else
                f32k_update4(hc0, lc0, hl, ll, hr, lr, hs, hn, hm0, hp0, ls, ln, lm0, lp0, d0, s0, nu2, h1, l1, d1);
            if (EXACT) l1 = lo_round4(h1, l1);
            if (RAGGED) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (xc[e] == 2) {  // the +x ghost: keeps level n (Dirichlet) or its Robin update
                        float a = el(hc0, e), b = el(lc0, e);
                        if (robin) {
                            const float2 ab = coef(B, 1, (long long)p * L.ny + y);
                            const float gi = e == 0 ? hl : el(hc0, e - 1), li = e == 0 ? ll : el(lc0, e - 1);
                            robin_update_f32k(ab.x, ab.y, el(hc0, e), el(lc0, e), gi, li, a, b);
                            if (EXACT) b = lo_round(a, b);
                        }
                        set(h1, e, a);
                        set(l1, e, b);
                        set(d1, e, el(d0, e));
                    }
            }
        } else if (robin && R.in) {
            // a z-face ghost plane (p = -1 or nz) of an interior row: the radiation update
            float4 gin = hm0, lgin = lm0;
            if (p < 0) {
                gin = lds4(Hs(it + 1) + sr * kFC + col);
                lgin = lo_decode4(gin, ldsl4(Ls(it + 1) + sr * kFC + col));
            }
            robin4(B, p < 0 ? 4 : 5, (long long)y * L.nx + xa, hc0, lc0, gin, lgin, h1, l1, nlive);
            if (EXACT) l1 = lo_round4(h1, l1);
        } else if (robin && R.ghost) {
            // a y-face ghost row at a plane of the tile: the radiation update from the interior row next to it
            const int si = y < 0 ? sr + 1 : sr - 1;
            const float4 gin = lds4(H + si * kFC + col);
            const float4 lgin = lo_decode4(gin, ldsl4(Lo + si * kFC + col));
            robin4(B, y < 0 ? 2 : 3, (long long)p * L.nx + xa, hc0, lc0, gin, lgin, h1, l1, nlive);
            if (EXACT) l1 = lo_round4(h1, l1);
        }
        *reinterpret_cast<float4*>(rh(it & 1, r, col)) = h1;
        *reinterpret_cast<float4*>(rl(it & 1, r, col)) = l1;
    };
    // the level-(n+2) y-face ghost row R at plane q (iteration it), from the level-(n+1) ghost row and its interior
    // neighbour row, both in ring slot (it - 1) & 1
    auto ghost_row2 = [&](const Row& R, int it) {
        const int q = k0 - 2 + it, slot = (it - 1) & 1;
        const int ri = R.y < 0 ? R.r + 1 : R.r - 1;
        const float4 hg = *reinterpret_cast<const float4*>(rh(slot, R.r, col));
        const float4 lg = *reinterpret_cast<const float4*>(rl(slot, R.r, col));
        const float4 gin = *reinterpret_cast<const float4*>(rh(slot, ri, col));
        const float4 lgin = *reinterpret_cast<const float4*>(rl(slot, ri, col));
        float4 ho, lo;
        robin4(B, R.y < 0 ? 2 : 3, (long long)q * L.nx + xa, hg, lg, gin, lgin, ho, lo, nlive);
        const long long qo = L.at(xa, R.y, q);
        if (!idx_ok(qo, nlive, L.elems, B.err)) return;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < nlive) {
                hi_n[qo + e] = el(ho, e);
                lo_n[qo + e] = lo_encode(el(ho, e), el(lo, e));
            }
    };

    if (warp == 0) {
        // ---------------- warp 0: the halo rows 0 and 9 ------------------------------------------------------------
        const Row R0 = make_row(0), R9 = make_row(kFR - 1);
        float4 hm[2] = {z4, z4}, lm[2] = {z4, z4}, hc[2] = {z4, z4}, lc[2] = {z4, z4};
        for (int it = 0; it < iters; ++it) {
            const int p = k0 - 1 + it, q = p - 1;
            const bool in_tile = p >= k0 && p < k1;
            bool ok = !*abort_flag;
            if (ok && (R0.live || R9.live)) ok = wait_stage(it);
            if (ok && in_tile && ((R0.in && p < L.nz) || (R9.in && p < L.nz))) ok = wait_stage(it + 1);
            ok = __all_sync(0xffffffffu, ok);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const Row& R = u ? R9 : R0;
                if (ok && R.live) {
                    hc[u] = lds4(Hs(it) + R.sr * kFC + col);
                    lc[u] = lo_decode4(hc[u], ldsl4(Ls(it) + R.sr * kFC + col));
                    if (in_tile) {  // the neighbouring rows' level n+2 needs these rows at the tile's planes only
                        float4 h1, l1, d1, s0;
                        level1(R, it, hm[u], lm[u], hc[u], lc[u], h1, l1, d1, s0);
                    }
                }
                if (ok && robin && R.ghost && it >= 1 && q >= k0 && q < k1) ghost_row2(R, it);
                hm[u] = hc[u];
                lm[u] = lc[u];
            }
            __syncthreads();
        }
        return;
    }

    // ---------------- warps 1..8 --------------------------------------------------------------------------------------
    const Row R = make_row(warp);
    float4 hm0 = z4, lm0 = z4, hc0 = z4, lc0 = z4;        // level n, own row: planes p-1, p
    float4 m1 = z4, lm1 = z4, c1 = z4, lc1 = z4;          // level n+1, own row: planes p-2, p-1
    float4 d1c = z4, sc = z4;                              // level-(n+1) increment and source at plane p-1
    // level n at plane k0-2 (not staged), needed when plane k0-1 is an interior plane of an interior row
    if (R.in && k0 >= 1 && xa <= L.nx) {
        const long long q = L.at(xa, R.y, k0 - 2);
        hm0 = __ldg(reinterpret_cast<const float4*>((const float*)A.hi_c + q));
        lm0 = lo_decode4(hm0, __ldg(reinterpret_cast<const uint2*>((const lo_t*)A.lo_c + q)));
    }

    for (int it = 0; it < iters; ++it) {
        const int p = k0 - 1 + it, q = p - 1;
        const bool in_tile = p >= k0 && p < k1;
        // interior rows need level n+1 at every plane k0-1 .. k1 (their own level n+2), a ghost row at the tile's
        const bool need1 = R.in || (R.ghost && in_tile);
        bool ok = !*abort_flag;
        if (ok && R.live) ok = wait_stage(it);
        if (ok && need1 && R.in && p < L.nz) ok = wait_stage(it + 1);
        ok = __all_sync(0xffffffffu, ok);
        float4 h1 = z4, l1 = z4, d1 = z4, s0 = z4;
        if (ok && R.live) {
            hc0 = lds4(Hs(it) + R.sr * kFC + col);
            lc0 = lo_decode4(hc0, ldsl4(Ls(it) + R.sr * kFC + col));
            if (need1) level1(R, it, hm0, lm0, hc0, lc0, h1, l1, d1, s0);
        }

        // ---- level n+2 at plane q = p-1 from level n+1 planes p-2 (m1), p-1 (c1), p (h1) ----
        if (ok && it >= 1) {
            const int slot = (it - 1) & 1, r = R.r, y = R.y;
            if (R.in && q >= k0 && q < k1) {
                const float4 ys = *reinterpret_cast<const float4*>(rh(slot, r - 1, col));
                const float4 yn = *reinterpret_cast<const float4*>(rh(slot, r + 1, col));
                const float4 lys = *reinterpret_cast<const float4*>(rl(slot, r - 1, col));
                const float4 lyn = *reinterpret_cast<const float4*>(rl(slot, r + 1, col));
                float gl = __shfl_up_sync(0xffffffffu, c1.w, 1), gll = __shfl_up_sync(0xffffffffu, lc1.w, 1);
                float gr = __shfl_down_sync(0xffffffffu, c1.x, 1), grl = __shfl_down_sync(0xffffffffu, lc1.x, 1);
                if (lane == 0) {
                    gl = *rh(slot, r, 3);
                    gll = *rl(slot, r, 3);
                }
                if (lane == 31) {
                    gr = *rh(slot, r, kFX + 4);
                    grl = *rl(slot, r, kFX + 4);
                }
                float4 ho, lo, dout;
                if (EXACT)
                    f32k_update4_scalar(c1, lc1, gl, gll, gr, grl, ys, yn, m1, h1, lys, lyn, lm1, l1, d1c, sc, nu2, ho,
                                        lo, dout);
                else
                    f32k_update4(c1, lc1, gl, gll, gr, grl, ys, yn, m1, h1, lys, lyn, lm1, l1, d1c, sc, nu2, ho, lo, dout);
                const long long qo = L.at(xa, y, q);
                if (!idx_ok(qo, 4, L.elems, B.err)) {
                } else if (!RAGGED || xa + 3 < L.nx) {
                    *reinterpret_cast<float4*>(hi_n + qo) = ho;
                    *reinterpret_cast<uint2*>(lo_n + qo) = lo_encode4(ho, lo);
                    *reinterpret_cast<float4*>(d_out + qo) = dout;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (xc[e] == 0) {
                            hi_n[qo + e] = el(ho, e);
                            lo_n[qo + e] = lo_encode(el(ho, e), el(lo, e));
                            d_out[qo + e] = el(dout, e);
                        } else if (xc[e] == 2 && robin) {  // the level-(n+2) +x ghost
                            const float2 ab = coef(B, 1, (long long)q * L.ny + y);
                            const float gi = e == 0 ? gl : el(c1, e - 1), li = e == 0 ? gll : el(lc1, e - 1);
                            float a, b;
                            robin_update_f32k(ab.x, ab.y, el(c1, e), el(lc1, e), gi, li, a, b);
                            hi_n[qo + e] = a;
                            lo_n[qo + e] = lo_encode(a, b);
                        }
                    }
                }
            } else if (robin && R.ghost && q >= k0 && q < k1) {
                ghost_row2(R, it);
            }
            // level-(n+2) z-face ghost planes: -1 (from level n+1 at -1 and 0), nz (from nz and nz-1)
            if (robin && R.in && (q == -1 || p == L.nz)) {
                const bool lo_face = q == -1;
                const float4 hg = lo_face ? c1 : h1, lg = lo_face ? lc1 : l1;
                const float4 hin = lo_face ? h1 : c1, lin = lo_face ? l1 : lc1;
                float4 ho, lo;
                robin4(B, lo_face ? 4 : 5, (long long)y * L.nx + xa, hg, lg, hin, lin, ho, lo, nlive);
                const long long qo = L.at(xa, y, lo_face ? -1 : L.nz);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < nlive && idx_ok(qo + e, 1, L.elems, B.err)) {
                        hi_n[qo + e] = el(ho, e);
                        lo_n[qo + e] = lo_encode(el(ho, e), el(lo, e));
                    }
            }
        }
        // shift the queues: level n (own row) and level n+1
        hm0 = hc0;
        lm0 = lc0;
        m1 = c1;
        lm1 = lc1;
        c1 = h1;
        lc1 = l1;
        d1c = d1;
        sc = s0;
        __syncthreads();
    }
}

__global__ void __maxnreg__(96)  // 2 blocks of 320 threads per SM (5 warps of 96 registers per SM quarter)
    k_temporal2_tma(const __grid_constant__ CUtensorMap m_hi, const __grid_constant__ CUtensorMap m_lo,
                    const __grid_constant__ CUtensorMap m_d, const __grid_constant__ CUtensorMap m_s,
                    const SweepArgs A, float* __restrict__ d_out, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_full[kFS];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFS; ++s) mbar_init(smem_addr(&bar_full[s]), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const bool ragged = (int)(blockIdx.x * kFX) + kFX > A.L.nx;
    if (A.exact) {
        if (ragged)
            fused2_block<true, true>(&m_hi, &m_lo, &m_d, &m_s, A, d_out, err, smem, bar_full, &abort_flag);
        else
            fused2_block<false, true>(&m_hi, &m_lo, &m_d, &m_s, A, d_out, err, smem, bar_full, &abort_flag);
    } else {
        if (ragged)
            fused2_block<true, false>(&m_hi, &m_lo, &m_d, &m_s, A, d_out, err, smem, bar_full, &abort_flag);
        else
            fused2_block<false, false>(&m_hi, &m_lo, &m_d, &m_s, A, d_out, err, smem, bar_full, &abort_flag);
    }
}

constexpr int kZ2 = 32;  // level-(n+2) planes per block

// tensor maps of the staged level-n state with this kernel's boxes: hi[0..1], lo[0..1], dlt[0..1], s
int tma2_maps(hg_grid* g) {
    if (g->tm2_ready) return HG_OK;
    const Layout& L = g->L;
    int rc;
    for (int b = 0; b < 2; ++b) {
        if ((rc = tma_encode(&g->tm2[0 + b], g->phi[b], L, 4, kFC, kFH))) return rc;
        if ((rc = tma_encode(&g->tm2[2 + b], g->lo[b], L, 2, kFC, kFH))) return rc;
        if ((rc = tma_encode(&g->tm2[4 + b], g->dlt[b], L, 4, kFC, kFR))) return rc;
    }
    if ((rc = tma_encode(&g->tm2[6], g->rho, L, 4, kFC, kFR))) return rc;
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
    if ((rc = smem_attr_once((const void*)k_temporal2_tma, F2::smem, &attr_done))) return rc;
    const int zb = g->zb > 0 ? (g->zb < g->nz ? g->zb : g->nz) : (g->nz < kZ2 ? g->nz : kZ2);
    SweepArgs A = sweep_args(g, zb);
    A.B.faces = g->bc == HG_BC_ROBIN ? 1 : 0;
    A.B.periodic = 0;
    A.B.xfaces = 0;
    const int c = g->cur;
    dim3 grid((g->nx + kFX - 1) / kFX, (g->ny + kFY - 1) / kFY, (g->nz + zb - 1) / zb);
    if ((rc = prof_begin(g))) return rc;
    k_temporal2_tma<<<grid, kFThreads, F2::smem, g->stream>>>(g->tm2[0 + c], g->tm2[2 + c], g->tm2[4 + g->dcur],
                                                              g->tm2[6], A, (float*)g->dlt[1 - g->dcur], g->derr);
    HG_LAUNCHED("TMA-staged depth-2 sub-step kernel");
    return prof_end(g);
}

}  // namespace hg
