// CPU check of the integer-pipe logarithm (emt_intlog.cuh): prints, for n
// pseudo-random arguments of each kind, the count that differ from the C
// library's log, and writes up to `keep` of them (argument, libm, integer
// path) for a high-precision comparison by the test.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2203_09467_gb300/csrc/emt_intlog.cuh"

static uint64_t g_s = 88172645463325252ull;
static uint64_t next()
{
    g_s ^= g_s << 13;
    g_s ^= g_s >> 7;
    g_s ^= g_s << 17;
    return g_s;
}
static uint64_t bits(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}
static double from_bits(uint64_t b)
{
    double x;
    memcpy(&x, &b, 8);
    return x;
}

int main(int argc, char** argv)
{
    const long n = argc > 1 ? atol(argv[1]) : 1000000;
    const long keep = argc > 2 ? atol(argv[2]) : 0;
    const char* path = argc > 3 ? argv[3] : nullptr;
    FILE* f = path ? fopen(path, "w") : nullptr;
    long diff = 0, big = 0, kept = 0;
    for (long i = 0; i < n; ++i) {
        const uint64_t w = next();
        double x;
        switch (i % 4) {
        case 0: x = (double)(2 * (w >> 12) + 1) * 0x1p-53; break;               // uniforms in (0, 1)
        case 1: x = 1.0 - (double)((w >> 20) + 1) * 0x1p-53; break;              // just below 1
        case 2: x = 1.0 + (double)((w >> 20) + 1) * 0x1p-52; break;              // just above 1
        default: x = from_bits((w >> 2) & 0x7FEFFFFFFFFFFFFFull | 0x0010000000000000ull); break;  // any positive normal
        }
        const double a = std::log(x), b = emt::intlog::log_rn(x);
        if (bits(a) != bits(b)) {
            ++diff;
            const long d = (long)(bits(a) - bits(b));
            if (d > 1 || d < -1) ++big;
            if (f && kept < keep) {
                fprintf(f, "%a %a %a\n", x, a, b);
                ++kept;
            }
        }
    }
    if (f) fclose(f);
    // the edges of every reduction interval (X = 0.75 + j 2^-8 and one unit
    // either side), of the [0.75, 1.5) normalisation, and 1 +- k units
    for (int j = 0; j <= 192; ++j) {
        const double X = 0.75 + j * 0x1p-8;
        for (int e = -3; e <= 3; e += 3) {
            const double c = std::ldexp(X, e);
            for (int k = -2; k <= 2; ++k) {
                const double x = from_bits(bits(c) + (uint64_t)(int64_t)k);
                const double a = std::log(x), b = emt::intlog::log_rn(x);
                if (bits(a) != bits(b)) {
                    ++diff;
                    const long d = (long)(bits(a) - bits(b));
                    if (d > 1 || d < -1) ++big;
                }
            }
        }
    }
    for (int k = -2000; k <= 2000; ++k) {
        const double x = from_bits(bits(1.0) + (uint64_t)(int64_t)k);
        const double a = std::log(x), b = emt::intlog::log_rn(x);
        if (bits(a) != bits(b)) {
            ++diff;
            const long d = (long)(bits(a) - bits(b));
            if (d > 1 || d < -1) ++big;
        }
    }
    // special arguments take the native log (or agree with it exactly)
    const double sp[] = {0.0, -0.0, 0x1p-1074, 0x1p-1022, 0x1.fffffffffffffp+1023, 1.0, -1.0, 1.0 / 0.0, -1.0 / 0.0,
                         0.0 / 0.0, 0.75, 1.5, 0x1.7ffffffffffffp+0, 0x1.8p-1, 0x1.fep-1, 0x1.01p+0, 2.0, 0.5};
    for (double x : sp) {
        const double a = std::log(x), b = emt::intlog::log_rn(x);
        if (bits(a) != bits(b) && !(a != a && b != b)) {
            const long d = (long)(bits(a) - bits(b));
            ++diff;
            if (d > 1 || d < -1 || (a != a) != (b != b)) ++big;
        }
    }
    printf("%ld %ld %ld\n", n, diff, big);
    return 0;
}
