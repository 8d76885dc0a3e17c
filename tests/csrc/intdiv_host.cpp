// CPU check of the integer-pipe division and square root (emt_intdiv.cuh)
// against the C division operator and sqrt, which are the IEEE-754 correctly
// rounded results.
// The FP32 reciprocal seed is moved by -3..+3 units of its last place
// (pseudo-randomly per call) to cover the GPU estimate's error.
#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cstdlib>

static uint64_t g_s[2];
static int g_seed_err = 0;
#define EMT_INTDIV_SEED_ERROR(k) (g_seed_err)
#include "../../paper_2203_09467_gb300/csrc/emt_intdiv.cuh"

using emt::intdiv::bitsd;
using emt::intdiv::dbits;

static uint64_t next()
{
    uint64_t a = g_s[0], b = g_s[1], r = a + b;
    b ^= a;
    g_s[0] = ((a << 55) | (a >> 9)) ^ b ^ (b << 14);
    g_s[1] = (b << 36) | (b >> 28);
    return r;
}

int main(int argc, char** argv)
{
    const long n = argc > 1 ? atol(argv[1]) : 1000000;
    const uint64_t seed = argc > 2 ? strtoull(argv[2], nullptr, 10) : 1;
    g_s[0] = 0x9E3779B97F4A7C15ull ^ (seed * 0xD1B54A32D192ED03ull);
    g_s[1] = 0x632BE59BD9B4E019ull + seed;
    const uint64_t kM = (1ull << 52) - 1;
    long bad = 0, fast = 0;
    for (long i = 0; i < n; ++i) {
        uint64_t a = next(), b = next();
        switch (i & 7) {
        case 1: b = (b & kM) | (1023ull << 52); break;                         // y in [1, 2)
        case 2: b = (1023ull << 52) | (next() & 0xF); break;                   // y just above a power of 2
        case 3: b = (1023ull << 52) | (kM - (next() & 0xF)); break;            // y just below 2
        case 4: a = (a & ~kM) | (b & kM); break;                               // equal significands
        case 5: a = (1023ull << 52) | (kM - (next() & 0xFF)); break;           // x just below 2
        case 6:                                                                // exponents near each other
            a = (a & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(923 + next() % 200) << 52);
            b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(923 + next() % 200) << 52);
            break;
        case 7:                                                                // exact quotients
            b = (b & 0x800FFFFFFFFFFFFFull & ~0xFFFFFFFFull) | ((uint64_t)(1000 + next() % 40) << 52);
            a = dbits(bitsd(b) * bitsd((1023ull << 52) | (next() & kM & ~0xFFFFFFFFFull)));
            break;
        default: break;
        }
        g_seed_err = (int)(next() % 7) - 3;
        const double x = bitsd(a), y = bitsd(b);
        const int ex = (int)((a >> 52) & 0x7FF), ey = (int)((b >> 52) & 0x7FF), er = ex - ey + 1023;
        if (!((unsigned)(ex - 1) >= 2046u || (unsigned)(ey - 1) >= 2046u || (unsigned)(er - 2) >= 2044u)) ++fast;
        const double q0 = x / y, q1 = emt::intdiv::div_rn(x, y);
        if (dbits(q0) != dbits(q1) && !(q0 != q0 && q1 != q1)) {
            if (bad < 5) printf("mismatch %a / %a: %a, integer path %a\n", x, y, q0, q1);
            ++bad;
        }
    }
    // square roots: any positive double, significands near 1 and 2, exact squares
    long sbad = 0;
    for (long i = 0; i < n; ++i) {
        uint64_t a = next() >> 1;
        switch (i & 3) {
        case 1: a = (a & kM) | (1023ull << 52); break;
        case 2: a = (1023ull << 52) | (kM - (next() & 0xFF)); break;
        case 3: {
            const double q = bitsd((uint64_t)(900 + next() % 240) << 52 | (next() & kM & ~0xFFFFFFFull));
            a = dbits(q * q);
            break;
        }
        default: break;
        }
        g_seed_err = (int)(next() % 7) - 3;
        const double x = bitsd(a), r0 = std::sqrt(x), r1 = emt::intdiv::sqrt_rn(x);
        if (dbits(r0) != dbits(r1) && !(r0 != r0 && r1 != r1)) {
            if (sbad < 5) printf("sqrt mismatch %a: %a, integer path %a\n", x, r0, r1);
            ++sbad;
        }
    }
    // special operands: zeros, subnormals, infinities, NaNs, the ends of the
    // normal range and quotients that overflow or underflow
    const double sp[] = {0.0, -0.0, 0x1p-1074, -0x1p-1074, 0x1p-1022, 0x1.fffffffffffffp-1023, 0x1.fffffffffffffp+1023,
                         -0x1.fffffffffffffp+1023, 1.0, -1.0, 3.0, 0x1p+1000, 0x1p-1000, 1.0 / 0.0, -1.0 / 0.0,
                         0.0 / 0.0, 0x1.8p-1070, 2.5e-310, 7.0};
    long xbad = 0;
    for (double x : sp)
        for (double y : sp) {
            const double q0 = x / y, q1 = emt::intdiv::div_rn(x, y);
            if (dbits(q0) != dbits(q1) && !(q0 != q0 && q1 != q1)) {
                printf("special mismatch %a / %a: %a, integer path %a\n", x, y, q0, q1);
                ++xbad;
            }
        }
    for (double x : sp) {
        const double r0 = std::sqrt(x), r1 = emt::intdiv::sqrt_rn(x);
        if (dbits(r0) != dbits(r1) && !(r0 != r0 && r1 != r1)) {
            printf("special sqrt mismatch %a: %a, integer path %a\n", x, r0, r1);
            ++xbad;
        }
    }
    printf("%ld %ld %ld\n", n, fast, bad + sbad + xbad);
    return bad + sbad + xbad != 0;
}
