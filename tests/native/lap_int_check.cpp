// Host check of the integer forms in lap_int.cuh (the Laplacian sum and 2c - prev) against the FP64 evaluation order
// they replace, compiled without contraction: prints "cases accepted mismatches" over seeded random inputs of several
// kinds (n sextuples through both Laplacian forms and n pairs).
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#include <stdint.h>

#include "../../paper_1602_05700_gb300/csrc/lap_int.cuh"

static double lap_fp64(double c, const double* x) {
    double L = (x[0] - c) + (x[1] - c);
    L = L + (x[2] - c);
    L = L + (x[3] - c);
    L = L + (x[4] - c);
    return L + (x[5] - c);
}

static uint64_t state;
static uint64_t next_u64() {  // splitmix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double unif() { return (double)(next_u64() >> 11) * 0x1.0p-53; }

int main(int argc, char** argv) {
    const long n = argc > 1 ? atol(argv[1]) : 1000000;
    state = argc > 2 ? strtoull(argv[2], 0, 10) : 1;
    long accepted = 0, mismatches = 0, cases = 0;
    for (long t = 0; t < n; ++t) {
        const int kind = (int)(next_u64() % 11);
        double c, x[6];
        // c: a potential-like value of either sign over many binades, sometimes at a power of two
        c = -(0.01 + unif()) * ldexp(1.0, (int)(next_u64() % 40) - 20);
        if (next_u64() % 4 == 0) c = -c;
        if (kind == 7) c = ldexp(1.0, (int)(next_u64() % 20) - 10) * (next_u64() % 2 ? 1 : -1);
        if (kind == 8) c = (1.0 + unif()) * ldexp(1.0, (int)(next_u64() % 2098) - 1075);  // any binade
        if (kind == 9) c = next_u64() % 8 ? 0.0 : (next_u64() % 2 ? -0.0 : 0x1p-1074 * (double)(next_u64() % 9));
        for (int i = 0; i < 6; ++i) {
            const double r = 2.0 * unif() - 1.0;
            switch (kind) {
                case 0: x[i] = c * (1.0 + 1e-3 * r); break;                       // smooth field
                case 1: x[i] = c * (1.0 + 1e-12 * r); break;                      // nearly flat
                case 2: x[i] = c * (1.0 + 0.9 * r); break;                        // rough: exponents e_c +- 1
                case 3: x[i] = next_u64() % 3 ? c : c * (1.0 + 1e-6 * r); break;  // exact ties and zeros
                case 4: x[i] = c * (1.0 + 3.0 * r); break;                        // exponents +- 2, sign changes
                case 5: x[i] = next_u64() % 5 ? c * (1.0 + 1e-4 * r) : (next_u64() % 2 ? 0.0 : -0.0); break;
                case 6: x[i] = hg::bits_d(hg::dbits(c) + (int64_t)(next_u64() % 2048) - 1024); break;  // ulps of c
                case 7: x[i] = c * (1.0 + ldexp(r, -(int)(next_u64() % 60))); break;          // near 2^50 units
                case 8: x[i] = hg::bits_d(hg::dbits(c) + (int64_t)(next_u64() % 64) - 32); break;
                case 10: x[i] = c * exp(0.8 * r); break;  // steep tail: neighbours up to a factor of 2.2 apart
                default: {  // quiet region ahead of a front: mostly +0, some -0, subnormals, small normals
                    const int w = (int)(next_u64() % 16);
                    x[i] = w < 11 ? 0.0 : w == 11 ? -0.0 : w == 12 ? 0x1p-1074 * (double)(next_u64() % 5)
                         : w == 13 ? -0x1p-1070 : ldexp(r, -(int)(next_u64() % 1100));
                }
            }
        }
        const double Lf = lap_fp64(c, x);
        for (int path = 0; path < 2; ++path) {  // exact-sum path; exact differences summed in FP64
            double Li = 0.0, d[6];
            bool ok;
            if (path == 0) {
                ok = hg::lap6_int(c, x[0], x[1], x[2], x[3], x[4], x[5], Li);
            } else {
                ok = hg::lap6_diffs(c, x[0], x[1], x[2], x[3], x[4], x[5], d);
                for (int i = 0; ok && i < 6; ++i)
                    if (hg::dbits(d[i]) != hg::dbits(x[i] - c)) {
                        if (mismatches < 5) fprintf(stderr, "difference %d: c=%a x=%a int=%a\n", i, c, x[i], d[i]);
                        ++mismatches;
                    }
                Li = ((((d[0] + d[1]) + d[2]) + d[3]) + d[4]) + d[5];
            }
            ++cases;
            if (!ok) continue;
            ++accepted;
            if (hg::dbits(Li) != hg::dbits(Lf)) {
                if (mismatches < 5)
                    fprintf(stderr, "mismatch path %d kind %d c=%a x=%a %a %a %a %a %a int=%a fp64=%a\n", path, kind, c,
                            x[0], x[1], x[2], x[3], x[4], x[5], Li, Lf);
                ++mismatches;
            }
        }
    }
    // 2c - prev: prev near c (smooth), exactly c, a few ulps away, up to and beyond 2|c|, of either sign, zeros
    for (long t = 0; t < n; ++t) {
        const int kind = (int)(next_u64() % 7);
        double c = -(0.01 + unif()) * ldexp(1.0, (int)(next_u64() % 40) - 20), p;
        if (next_u64() % 4 == 0) c = -c;
        if (kind == 6) c = (1.0 + unif()) * ldexp(1.0, (int)(next_u64() % 2098) - 1075);
        const double r = 2.0 * unif() - 1.0;
        switch (kind) {
            case 0: p = c * (1.0 + 1e-3 * r); break;
            case 1: p = c; break;
            case 2: p = hg::bits_d(hg::dbits(c) + (int64_t)(next_u64() % 64) - 32); break;
            case 3: p = c * (1.0 + 1.2 * r); break;
            case 4: p = c * 2.0 * (1.0 + ldexp(r, -(int)(next_u64() % 54))); break;
            case 5: c = next_u64() % 2 ? 0.0 : c; p = next_u64() % 2 ? 0.0 : (next_u64() % 2 ? -0.0 : 0x1p-1074); break;
            default: p = hg::bits_d(hg::dbits(c) + (int64_t)(next_u64() % 4096) - 2048); break;
        }
        double ti = 0.0;
        const bool ok = hg::twice_minus_int(c, p, ti);
        ++cases;
        if (!ok) continue;
        ++accepted;
        const double tf = 2.0 * c - p;
        if (hg::dbits(ti) != hg::dbits(tf)) {
            if (mismatches < 5) fprintf(stderr, "2c-prev mismatch kind %d c=%a p=%a int=%a fp64=%a\n", kind, c, p, ti, tf);
            ++mismatches;
        }
    }
    printf("%ld %ld %ld\n", cases, accepted, mismatches);
    return 0;
}
