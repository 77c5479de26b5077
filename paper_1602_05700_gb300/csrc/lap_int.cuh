// The FP64 Laplacian sum of the sub-step, L = (((((xl-c) + (xr-c)) + (ys-c)) + (yn-c)) + (zm-c)) + (zp-c) with
// every difference and every partial sum rounded to double (the plain evaluation order of Eq. HNeq's discretisation,
// Sec. 2), computed with integer instructions where no rounding of that order changes anything.
//
// Why: GB300 executes FP64 arithmetic at about 2 operations per SM per clock, while its integer pipes take 64 lanes
// per clock; the 11 FP64 operations of L are most of an FP64 sub-step's 15.  When they are all exact, their result is
// the exact sum of the six differences, which integers give bit for bit.
//
// When every operation is exact: write each value as sign * M * 2^(e - 1075) (M the 53-bit significand, e the biased
// exponent).  If c is normal with 64 <= e_c <= 2000 and each neighbour x has c's sign and an exponent within one of
// e_c, then |x| and |c| are integers X, C in units u = 2^(e_c - 1 - 1075), and x - c = sgn(c) (X - C) u exactly.  If
// also |X - C| < 2^50 for all six, every difference and every partial sum is an integer below 6 * 2^50 < 2^53 in
// units of u (u >= 2^-1012, a normal number), hence representable: IEEE subtraction and addition return them
// exactly, and L = sgn(c) S u with S the integer sum (an exact zero being +0, as x - x and a + (-a) are in
// round-to-nearest).  A cell and six neighbours that are all +0 give L = +0 as well.  Otherwise lap6_int returns
// false and the caller evaluates the FP64 order itself.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif
#ifndef __CUDA_ARCH__
#include <string.h>
#endif

namespace hg {

constexpr unsigned long long kFrac52 = (1ull << 52) - 1;
constexpr unsigned long long kHidden52 = 1ull << 52;

__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    memcpy(&u, &x, sizeof u);
    return u;
#endif
}

__host__ __device__ __forceinline__ double bits_d(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
#endif
}

__host__ __device__ __forceinline__ int clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// The steep regions (neighbours up to a factor of 2 from c, as in the tails of a compact source) fail the 2^50 bound,
// but there each difference x - c is still exact (Sterbenz: c/2 <= x <= 2c of one sign), only the partial sums
// round: the six differences come from integers -- the same units, the bound replaced by the Sterbenz condition
// 2X >= C and X <= 2C -- and only the five additions remain for the FP64 unit.
//
// lap6_exact_sum evaluates the first condition (every operation of L exact; its S is then L in units of u) and
// lap6_exact_diffs the second (every difference exact), each in one pass over the six neighbours.  A stencil that
// passes the first passes the second, and a stencil of seven +0 passes both (L = +0, every difference +0).
struct Lap6Sum {
    long long S;  // sum of the six differences in units u = 2^(e_c - 1076), meaningful when exact
    bool exact;
};

__host__ __device__ __forceinline__ long long lap_units(double x, unsigned hc, long long C, unsigned& d) {
    const unsigned long long xb = dbits(x);
    d = (unsigned)(xb >> 52) - hc + 1u;  // 0, 1, 2: c's sign and exponent e_c - 1 .. e_c + 1
    return (long long)(((xb & kFrac52) | kHidden52) << (d & 3u));
}

// c normal in the range above, or c = +0 with six +0 neighbours (c = +0: its terms pass only for neighbours +0,
// D = 0, or positive subnormals, D > 0, so S = 0 means every neighbour is +0 -- the quiet regions ahead of a front)
__host__ __device__ __forceinline__ bool lap_c_ok(unsigned long long cb, long long S) {
    const unsigned ec = (unsigned)(cb >> 52) & 0x7ffu;
    return (ec >= 64u && ec <= 2000u) || (cb == 0ull && S == 0);
}

__host__ __device__ __forceinline__ Lap6Sum lap6_exact_sum(double c, double x0, double x1, double x2, double x3,
                                                           double x4, double x5) {
    const unsigned long long cb = dbits(c);
    const unsigned hc = (unsigned)(cb >> 52);  // sign and biased exponent of c
    const long long C = (long long)(((cb & kFrac52) | kHidden52) << 1);
    const double x[6] = {x0, x1, x2, x3, x4, x5};
    bool ok = true;
    long long S = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned d;
        const long long D = lap_units(x[i], hc, C, d) - C;
        ok = ok && d <= 2u && (unsigned long long)(D + (1ll << 50)) < (1ull << 51);
        S += D;
    }
    return {S, ok && lap_c_ok(cb, S)};
}

__host__ __device__ __forceinline__ bool lap6_exact_diffs(double c, double x0, double x1, double x2, double x3,
                                                          double x4, double x5) {
    const unsigned long long cb = dbits(c);
    const unsigned hc = (unsigned)(cb >> 52);
    const long long C = (long long)(((cb & kFrac52) | kHidden52) << 1);
    const double x[6] = {x0, x1, x2, x3, x4, x5};
    bool ok = true;
    long long S = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned d;
        const long long X = lap_units(x[i], hc, C, d);
        ok = ok && d <= 2u && 2 * X >= C && X <= 2 * C;
        S += X - C;
    }
    return ok && lap_c_ok(cb, S);
}

// S u with u = 2^(e_c - 1076), |S| < 2^54 with at most 53 significant bits: |S| = mant 2^-(lz - 11), mant in
// [2^52, 2^53), biased exponent e_c + 10 - lz; the sign is c's times S's; 0 gives +0
__host__ __device__ __forceinline__ double pack_units(long long S, double c) {
    const unsigned long long cb = dbits(c);
    const unsigned ec = (unsigned)(cb >> 52) & 0x7ffu;
    const unsigned long long A = (unsigned long long)(S < 0 ? -S : S);
    const int lz = clz64(A);
    const int sh = 11 - lz;
    const unsigned long long mant = sh > 0 ? A >> sh : A << ((-sh) & 63);
    const unsigned long long sign = (cb ^ (S < 0 ? (1ull << 63) : 0ull)) & (1ull << 63);
    return A == 0 ? 0.0 : bits_d(sign | ((((unsigned long long)(ec + 10u - (unsigned)lz) - 1ull) << 52) + mant));
}

// x - c from integers (valid when the stencil passed exact_diffs)
__host__ __device__ __forceinline__ double lap_diff(double x, double c) {
    const unsigned long long cb = dbits(c);
    unsigned d;
    const long long C = (long long)(((cb & kFrac52) | kHidden52) << 1);
    return pack_units(lap_units(x, (unsigned)(cb >> 52), C, d) - C, c);
}

// L from integers; false when some operation of the FP64 order might round (then L is not set)
__host__ __device__ __forceinline__ bool lap6_int(double c, double x0, double x1, double x2, double x3, double x4,
                                                  double x5, double& L) {
    const Lap6Sum k = lap6_exact_sum(c, x0, x1, x2, x3, x4, x5);
    if (k.exact) L = pack_units(k.S, c);
    return k.exact;
}

// the six differences from integers, in one pass; false (d not set) unless every difference is exact
__host__ __device__ __forceinline__ bool lap6_diffs(double c, double x0, double x1, double x2, double x3, double x4,
                                                    double x5, double (&d)[6]) {
    const unsigned long long cb = dbits(c);
    const unsigned hc = (unsigned)(cb >> 52);
    const long long C = (long long)(((cb & kFrac52) | kHidden52) << 1);
    const double x[6] = {x0, x1, x2, x3, x4, x5};
    bool ok = true;
    long long D[6], S = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned e;
        const long long X = lap_units(x[i], hc, C, e);
        ok = ok && e <= 2u && 2 * X >= C && X <= 2 * C;
        D[i] = X - C;
        S += D[i];
    }
    ok = ok && lap_c_ok(cb, S);
    if (ok) {
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = pack_units(D[i], c);
    }
    return ok;
}

// t = 2c - prev rounded once to nearest-even (the leapfrog's first operation), from integers where c is normal in the
// range above and prev has c's sign, an exponent within one of c's and |prev| < 2|c|: in units u = 2^(e_c - 1076),
// T = 4 M_c - M_prev 2^(e_prev - e_c + 1) is a positive integer below 2^55, rounded here to 53 significant bits.
// c = prev = +0 gives +0.  Otherwise false (t not set).
__host__ __device__ __forceinline__ bool twice_minus_int(double c, double prev, double& t) {
    const unsigned long long cb = dbits(c), pb = dbits(prev);
    const unsigned hc = (unsigned)(cb >> 52);
    const unsigned ec = hc & 0x7ffu;
    const unsigned d = (unsigned)(pb >> 52) - hc + 1u;
    const long long T = (long long)(((cb & kFrac52) | kHidden52) << 2) -
                        (long long)(((pb & kFrac52) | kHidden52) << (d & 3u));
    const unsigned long long Tu = (unsigned long long)T;
    const int k = 11 - clz64(Tu);  // significant bits beyond 53 (negative: room to shift left)
    unsigned long long q;
    if (k > 0) {
        const unsigned long long rem = Tu & ((1ull << k) - 1), half = 1ull << (k - 1);
        q = Tu >> k;
        q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;  // q = 2^53 carries into the exponent
    } else {
        q = Tu << ((-k) & 63);
    }
    const unsigned long long e = (unsigned long long)((int)ec + k - 1);  // biased exponent of the result
    t = (cb | pb) == 0ull ? 0.0 : bits_d((cb & (1ull << 63)) | (((e - 1ull) << 52) + q));
    return (cb | pb) == 0ull || (d <= 2u && T > 0 && ec >= 64u && ec <= 2000u);
}

}  // namespace hg
