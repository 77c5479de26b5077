// Per-cell arithmetic of one sub-step, shared by the single-sweep and the temporally blocked kernels so that both
// round identically (every operation is an explicit round-to-nearest intrinsic: no contraction choices are left
// to the compiler).  arXiv 1602.05700, Sec. 1 Eq. HNeq., discretised as
//   phi^{n+1} = 2 phi^n - phi^{n-1} + nu^2 sum_{6 nb}(phi^n_nb - phi^n) - s,  s = (c_h dt)^2 4 pi G (rho - rho_bar),
// where s is the stored source (scaled once, in FP64, when the density is set).
// The Laplacian is always summed as differences phi_nb - phi (exact for neighbouring values of similar size), never
// as sum(phi_nb) - 6 phi: the latter carries an error of order eps |phi| per sub-step, which the lossless scheme
// accumulates in its slow modes (about 3e-12 relative after 2000 sub-steps at 64^3 against ~3e-14).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lap_int.cuh"

namespace hg {

// ---- storage of the compensation -------------------------------------------------------------------------------
// The compensated state keeps phi^n = hi + lo with |lo| <= ulp(hi)/2 (lo is the exact rounding error of the
// Fast2Sum that produced hi).  lo is stored in 16 bits as the half-precision number f = 2^24 lo / hi, |f| <= 1, and
// read back as lo = hi (f 2^-24).  The code keeps 11 significant bits of lo, so phi is held to about 2^-36 |phi|
// (36 bits) instead of 48 -- far below the other float roundings of the sub-step (the FP32 source and increment),
// which set the accuracy -- for 2 bytes per cell instead of 4.  Every reader decodes a stored code to the same
// float (one rounded product), so all kernels see one and the same state.
using lo_t = __half;

__device__ __forceinline__ float lo_decode(float hi, lo_t f) {
    return __fmul_rn(hi, __fmul_rn(__half2float(f), 5.9604644775390625e-8f));  // f * 2^-24 is exact
}

// f = 2^24 lo / hi with the hardware's approximate reciprocal (rcp.approx: the code only has to be decoded
// consistently, so its last bits need no correct rounding); lo = 0 whenever hi = 0 (a Fast2Sum with a zero sum has a
// zero error), which the select keeps away from 0 * inf.  A nonzero lo never comes with a subnormal hi (a sum that
// rounds to a subnormal is exact), so |f| <= 1 (1 + 2^-22 with the approximate reciprocal).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ lo_t lo_encode(float hi, float lo) {
    const float f = lo == 0.f ? 0.f : __fmul_rn(__fmul_rn(lo, 16777216.f), rcp_approx(hi));
    return __float2half_rn(f);
}

// the value of lo after a store and a load (temporally blocked levels that never pass through memory use it to
// round exactly like the single sweep)
__device__ __forceinline__ float lo_round(float hi, float lo) { return lo_decode(hi, lo_encode(hi, lo)); }

// ---- packed pairs ---------------------------------------------------------------------------------------------
// sm_100 and later round two float operations in one instruction (add.f32x2, mul.f32x2, fma.f32x2), each exactly as
// the scalar operation would: the four-cell helpers below give the bits of four scalar calls in fewer instructions.
__device__ __forceinline__ float2 pa(const float4& v) { return make_float2(v.x, v.y); }  // cells 0, 1 of a group
__device__ __forceinline__ float2 pb(const float4& v) { return make_float2(v.z, v.w); }  // cells 2, 3
__device__ __forceinline__ float4 join4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// four consecutive codes as one 8-byte word
__device__ __forceinline__ float4 lo_decode4(const float4& hi, uint2 raw) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    const float2 k = dup2(5.9604644775390625e-8f);
    return join4(mul2(pa(hi), mul2(a, k)), mul2(pb(hi), mul2(b, k)));
}
__device__ __forceinline__ uint2 lo_encode4(const float4& hi, const float4& lo) {
    const float2 k = dup2(16777216.f);
    float2 fa = mul2(mul2(pa(lo), k), make_float2(rcp_approx(hi.x), rcp_approx(hi.y)));
    float2 fb = mul2(mul2(pb(lo), k), make_float2(rcp_approx(hi.z), rcp_approx(hi.w)));
    fa.x = lo.x == 0.f ? 0.f : fa.x;
    fa.y = lo.y == 0.f ? 0.f : fa.y;
    fb.x = lo.z == 0.f ? 0.f : fb.x;
    fb.y = lo.w == 0.f ? 0.f : fb.y;
    const __half2 ha = __floats2half2_rn(fa.x, fa.y), hb = __floats2half2_rn(fb.x, fb.y);
    uint2 r;
    r.x = *reinterpret_cast<const unsigned*>(&ha);
    r.y = *reinterpret_cast<const unsigned*>(&hb);
    return r;
}
// lo after a store and a load, for four cells
__device__ __forceinline__ float4 lo_round4(const float4& hi, const float4& lo) { return lo_decode4(hi, lo_encode4(hi, lo)); }

// f32 with compensated increments: phi^n = hi + lo, d = phi^n - phi^{n-1}.
//   L  = sum(hi_nb - hi) + sum(lo_nb) - 6 lo          (neighbour order -x, +x, -y, +y, -z, +z)
//   d' = d + (nu^2 L - s)
//   (hi', lo') = Fast2Sum(hi, lo + d')
__device__ __forceinline__ void f32k_update(float xl, float xr, float ys, float yn, float zm, float zp, float c,
                                            float lxl, float lxr, float lys, float lyn, float lzm, float lzp, float lc,
                                            float d, float s, float nu2, float& hi_o, float& lo_o, float& d_o) {
    float Lh = __fadd_rn(__fsub_rn(xl, c), __fsub_rn(xr, c));
    Lh = __fadd_rn(Lh, __fsub_rn(ys, c));
    Lh = __fadd_rn(Lh, __fsub_rn(yn, c));
    Lh = __fadd_rn(Lh, __fsub_rn(zm, c));
    Lh = __fadd_rn(Lh, __fsub_rn(zp, c));
    float Ll = __fadd_rn(__fadd_rn(__fadd_rn(lxl, lxr), __fadd_rn(lys, lyn)), __fadd_rn(lzm, lzp));
    Ll = __fmaf_rn(-6.0f, lc, Ll);
    const float inc = __fmaf_rn(nu2, __fadd_rn(Lh, Ll), -s);
    const float dn = __fadd_rn(d, inc);
    const float y = __fadd_rn(dn, lc);
    const float t = __fadd_rn(c, y);
    lo_o = __fsub_rn(y, __fsub_rn(t, c));
    hi_o = t;
    d_o = dn;
}

// The same sub-step for a group of four consecutive cells of a row (c, lc; x neighbours xl, lxl before the group
// and xr, lxr after it), written on packed pairs; operation for operation it is four f32k_update calls.  The x differences are shared between neighbouring
// cells: with D_e = c_{e+1} - c_e rounded (c_{-1} = xl, c_4 = xr), RN(c_{e-1} - c_e) = -D_{e-1} exactly, so the first
// partial sum (xl - c) + (xr - c) of cell e is RN(D_e - D_{e-1}); everything after it runs on packed pairs.
__device__ __forceinline__ void f32k_update4(const float4& c, const float4& lc, float xl, float lxl, float xr,
                                             float lxr, const float4& ys, const float4& yn, const float4& zm,
                                             const float4& zp, const float4& lys, const float4& lyn, const float4& lzm,
                                             const float4& lzp, const float4& d, const float4& s, float nu2,
                                             float4& ho, float4& lo, float4& dout) {
    const float Dm = __fsub_rn(c.x, xl), D0 = __fsub_rn(c.y, c.x), D1 = __fsub_rn(c.z, c.y), D2 = __fsub_rn(c.w, c.z),
                D3 = __fsub_rn(xr, c.w);
    const float2 n2 = dup2(nu2);
    // one pair after the other (cells 0, 1 then 2, 3), which keeps fewer values live at once
    auto pair = [&](float2 A, float2 L, float2 cc, float2 vys, float2 vyn, float2 vzm, float2 vzp, float2 lsy,
                    float2 lny, float2 lzmm, float2 lzpp, float2 lcc, float2 dd, float2 ss, float2& h2, float2& l2,
                    float2& d2) {
        A = add2(A, sub2(vys, cc));
        A = add2(A, sub2(vyn, cc));
        A = add2(A, sub2(vzm, cc));
        A = add2(A, sub2(vzp, cc));
        L = add2(add2(L, add2(lsy, lny)), add2(lzmm, lzpp));
        L = fma2(dup2(-6.0f), lcc, L);
        d2 = add2(dd, fma2(n2, add2(A, L), make_float2(-ss.x, -ss.y)));
        const float2 y = add2(d2, lcc);
        h2 = add2(cc, y);
        l2 = sub2(y, sub2(h2, cc));
    };
    float2 ha, la, da, hb, lb, db;
    pair(make_float2(__fsub_rn(D0, Dm), __fsub_rn(D1, D0)), make_float2(__fadd_rn(lxl, lc.y), __fadd_rn(lc.x, lc.z)),
         pa(c), pa(ys), pa(yn), pa(zm), pa(zp), pa(lys), pa(lyn), pa(lzm), pa(lzp), pa(lc), pa(d), pa(s), ha, la, da);
    pair(make_float2(__fsub_rn(D2, D1), __fsub_rn(D3, D2)), make_float2(__fadd_rn(lc.y, lc.w), __fadd_rn(lc.z, lxr)),
         pb(c), pb(ys), pb(yn), pb(zm), pb(zp), pb(lys), pb(lyn), pb(lzm), pb(lzp), pb(lc), pb(d), pb(s), hb, lb, db);
    ho = join4(ha, hb);
    lo = join4(la, lb);
    dout = join4(da, db);
}

// The same four cells by four scalar f32k_update calls.  The single sweep, the batched sweep and the fused kernels
// in exact mode use this form, so that they round identically to one another (one cell of a 2.4-million-update
// periodic run came out one unit in the last place apart between the packed and the scalar form inside the sweep
// kernel, although the two agree on every input tried in isolation; the exact modes therefore keep to one form).
__device__ __forceinline__ void f32k_update4_scalar(const float4& c, const float4& lc, float xl, float lxl, float xr,
                                                    float lxr, const float4& ys, const float4& yn, const float4& zm,
                                                    const float4& zp, const float4& lys, const float4& lyn,
                                                    const float4& lzm, const float4& lzp, const float4& d,
                                                    const float4& s, float nu2, float4& ho, float4& lo,
                                                    float4& dout) {
    f32k_update(xl, c.y, ys.x, yn.x, zm.x, zp.x, c.x, lxl, lc.y, lys.x, lyn.x, lzm.x, lzp.x, lc.x, d.x, s.x, nu2, ho.x,
                lo.x, dout.x);
    f32k_update(c.x, c.z, ys.y, yn.y, zm.y, zp.y, c.y, lc.x, lc.z, lys.y, lyn.y, lzm.y, lzp.y, lc.y, d.y, s.y, nu2,
                ho.y, lo.y, dout.y);
    f32k_update(c.y, c.w, ys.z, yn.z, zm.z, zp.z, c.z, lc.y, lc.w, lys.z, lyn.z, lzm.z, lzp.z, lc.z, d.z, s.z, nu2,
                ho.z, lo.z, dout.z);
    f32k_update(c.z, xr, ys.w, yn.w, zm.w, zp.w, c.w, lc.z, lxr, lys.w, lyn.w, lzm.w, lzp.w, lc.w, d.w, s.w, nu2, ho.w,
                lo.w, dout.w);
}

// f64: phi^{n+1} = ((2c - prev) + nu^2 L) - s with L = (((((xl-c) + (xr-c)) + (ys-c)) + (yn-c)) + (zm-c)) + (zp-c):
// each operation rounded separately, in this order -- the plain evaluation of the update.  Every FP64 rounding of
// the step is thereby fixed by the formula alone, so any IEEE implementation that evaluates it in the same order
// without contraction produces the same bits.  2c is exact, so 2c - prev is one fused multiply-add with the same
// single rounding: 15 FP64 instructions, of which L takes 11.  Where none of L's 11 operations rounds (the neighbours
// share c's sign, lie within a binade of it and differ from it by less than 2^50 of its half-ulps -- any smooth
// field, and the all-zero stencils ahead of a wave front), L is the integer sum of the six differences (lap_int.cuh,
// lap6_exact_sum / pack_units) with the same bits; where they differ more but each difference is still exact
// (neighbours within a factor of 2 of c, as in the steep tails of a compact source), the six differences come from
// integers (lap_diff) and only the five additions run in FP64; where prev has c's sign, lies within a binade of it
// and below 2|c|, twice_minus_int rounds 2c - prev from integers.  That leaves 3 FP64 instructions per cell in smooth
// regions (nu^2 L, the add, the subtraction of s); outside those conditions the FP64 operations run as written.
__device__ __forceinline__ double lap6_fp64(double xl, double xr, double ys, double yn, double zm, double zp,
                                            double c) {
    double L = __dadd_rn(__dsub_rn(xl, c), __dsub_rn(xr, c));
    L = __dadd_rn(L, __dsub_rn(ys, c));
    L = __dadd_rn(L, __dsub_rn(yn, c));
    L = __dadd_rn(L, __dsub_rn(zm, c));
    return __dadd_rn(L, __dsub_rn(zp, c));
}

// Out-of-line FP64 forms for the per-lane choice: a lane that needs one calls it, and the common path carries none
// of its FP64 instructions.
static __device__ __noinline__ double sum6_ool(double d0, double d1, double d2, double d3, double d4, double d5) {
    return __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(d0, d1), d2), d3), d4), d5);
}
static __device__ __noinline__ double lap6_ool(double xl, double xr, double ys, double yn, double zm, double zp,
                                               double c) {
    return lap6_fp64(xl, xr, ys, yn, zm, zp, c);
}
static __device__ __noinline__ double twice_minus_ool(double c, double prev) { return __fma_rn(2.0, c, -prev); }

// WARP_UNIFORM: the form is chosen per warp (the cheapest form every lane of the warp can take), so that a warp never
// executes two forms one after the other -- the batched launches, whose small grids mix the forms within a warp;
// otherwise per lane, the slower forms out of line -- the single-grid sweep, measured faster that way on a 512^3
// grid.  Each form gives every lane the same bits.
template <bool WARP_UNIFORM>
__device__ __forceinline__ double f64_update(double xl, double xr, double ys, double yn, double zm, double zp, double c,
                                             double prev, double s, double nu2) {
    double L, t;
    const Lap6Sum k = lap6_exact_sum(c, xl, xr, ys, yn, zm, zp);
    if (WARP_UNIFORM) {
        const unsigned m = __activemask();
        if (__all_sync(m, k.exact)) {
            L = pack_units(k.S, c);
        } else if (__all_sync(m, lap6_exact_diffs(c, xl, xr, ys, yn, zm, zp))) {
            L = __dadd_rn(lap_diff(xl, c), lap_diff(xr, c));
            L = __dadd_rn(L, lap_diff(ys, c));
            L = __dadd_rn(L, lap_diff(yn, c));
            L = __dadd_rn(L, lap_diff(zm, c));
            L = __dadd_rn(L, lap_diff(zp, c));
        } else {
            L = lap6_fp64(xl, xr, ys, yn, zm, zp, c);
        }
        const bool ti = twice_minus_int(c, prev, t);
        if (!__all_sync(m, ti)) t = __fma_rn(2.0, c, -prev);
    } else {
        if (k.exact) {
            L = pack_units(k.S, c);
        } else {
            double d[6];
            if (lap6_diffs(c, xl, xr, ys, yn, zm, zp, d))
                L = sum6_ool(d[0], d[1], d[2], d[3], d[4], d[5]);
            else
                L = lap6_ool(xl, xr, ys, yn, zm, zp, c);
        }
        if (!twice_minus_int(c, prev, t)) t = twice_minus_ool(c, prev);
    }
    return __dsub_rn(__dadd_rn(t, __dmul_rn(nu2, L)), s);
}

// Robin ghost sub-step in FP64 (monopole radiation condition, upwinded) for u = r phi:
// u_g' = u_g - a (u_g - u_i), phi_g' = u_g' / r_g, with a = nu / mu, in that order of operations
__device__ __forceinline__ double robin_update_f64(double a, double rg, double ri, double phi_g, double phi_i) {
    const double ug = __dmul_rn(rg, phi_g), ui = __dmul_rn(ri, phi_i);
    return __ddiv_rn(__dsub_rn(ug, __dmul_rn(a, __dsub_rn(ug, ui))), rg);
}

// The same update for the compensated float state, written phi_g' = alpha phi_g + beta phi_i (alpha = 1 - a,
// beta = a r_i / r_g), without FP64 (GB300's FP64 and its f32<->f64 conversions are slow): alpha, beta rounded to
// float; both products and their sum carried as float pairs by error-free
// transformations (TwoProduct with an FMA, TwoSum), the compensations added, then one Fast2Sum.
__device__ __forceinline__ void robin_update_f32k(float a, float b, float hg, float lg, float hin, float lin,
                                                  float& hi_o, float& lo_o) {
    const float p1 = __fmul_rn(a, hg);
    const float e1 = __fmaf_rn(a, hg, -p1);
    const float p2 = __fmul_rn(b, hin);
    const float e2 = __fmaf_rn(b, hin, -p2);
    const float s = __fadd_rn(p1, p2);
    const float bv = __fsub_rn(s, p1);
    const float e3 = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bv)), __fsub_rn(p2, bv));
    float t = __fadd_rn(__fadd_rn(e1, e2), e3);
    t = __fmaf_rn(a, lg, t);
    t = __fmaf_rn(b, lin, t);
    hi_o = __fadd_rn(s, t);
    lo_o = __fsub_rn(t, __fsub_rn(hi_o, s));
}

// a double as a float and the code of its rounding remainder, and back
__device__ __forceinline__ void split_f32(double v, float& hi, lo_t& lo) {
    hi = __double2float_rn(v);
    // a subnormal (or zero) hi keeps no compensation: its remainder is below 2^-149 and has no code
    lo = lo_encode(hi, fabsf(hi) < 1.17549435e-38f ? 0.f : __double2float_rn(__dsub_rn(v, (double)hi)));
}
__device__ __forceinline__ double join_f32(float hi, lo_t lo) {
    return __dadd_rn((double)hi, (double)lo_decode(hi, lo));
}

}  // namespace hg
