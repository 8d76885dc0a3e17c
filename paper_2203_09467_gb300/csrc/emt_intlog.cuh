// emt_intlog.cuh -- natural logarithm of an FP64 value on the integer pipe.
//
// GB300 runs FP64 at 1/64 of its FP32 rate; a polynomial logarithm in FP64
// occupies that narrow pipe for tens of instructions, and one is taken in
// every step (the free path -ln u).  `log_rn(x)` forms ln x in 128-bit
// fixed point from the integer significand and exponent of x:
//   x = 2^E X, X in [0.75, 1.5);  ln x = E ln 2 + ln(1 / c_j) + ln(1 + r),
// c_j = I_j 2^-15 a 16-bit reduction factor chosen by the top bits of X
// (table emt_logtab.h, exact values from gen_logtab.py; c_j = 1 next to
// X = 1), r = X c_j - 1 formed exactly as an integer multiple of 2^-68
// (|r| <= 2^-8), and
//   ln(1 + r) = r - r^2/2 + r^3 P3(r),  P3(r) = sum_{n=0..6} (-r)^n / (n + 3)
// (Taylor series; the first two terms exact in 128 bits, r^2 P3 in units of
// 2^-78, so the error is below 2^-77 of ln(1 + r)).  The sum is a signed
// multiple of 2^-116 (2^-128 next to x = 1, where the result is ln(1 + r)
// alone and may be tiny) and is rounded once to the nearest double.  The
// result is the correctly rounded logarithm except when ln x lies within
// about 2^-75 (relative) of a rounding boundary.  On 4e6 random arguments
// (uniforms, both sides of 1, any positive normal) it differs from the C
// library's log in 2.1e-4 of them, by one unit in the last place, and a
// 240-bit reference sides with it in every one of those cases.  Arguments
// x = 1 - k 2^-53 with small k are such exceptions: their logarithm lies
// within 1e-11 units of a midpoint, finer than the fixed-point sum.  Non-positive, subnormal and
// non-finite arguments take the native log.
#pragma once

#include <stdint.h>
#include <string.h>

#include "emt_logtab.h"

#if defined(__CUDACC__)
#define EMT_LHD __host__ __device__ __forceinline__
#define EMT_LHD_CALL static __host__ __device__ __noinline__  // one copy per kernel (instruction cache)
#else
#define EMT_LHD static inline
#define EMT_LHD_CALL static inline
#endif

namespace emt {
namespace intlog {

typedef unsigned __int128 u128;
typedef __int128 i128;

#if defined(__CUDACC__)
static __device__ const uint32_t d_inv[192] = EMT_LOGTAB_INV;
static __device__ const uint64_t d_thi[192] = EMT_LOGTAB_HI;
static __device__ const uint64_t d_tlo[192] = EMT_LOGTAB_LO;
#endif
static const uint32_t h_inv[192] = EMT_LOGTAB_INV;
static const uint64_t h_thi[192] = EMT_LOGTAB_HI;
static const uint64_t h_tlo[192] = EMT_LOGTAB_LO;

EMT_LHD int clz64(uint64_t v)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// floor((a b) / 2^64) for signed a, b
EMT_LHD int64_t mulhi(int64_t a, int64_t b) { return (int64_t)(((i128)a * b) >> 64); }

// Q0.64 coefficients 1/(n + 3), n = 0..6, rounded to nearest
constexpr int64_t kC3 = 6148914691236517205ll;
constexpr int64_t kC4 = 4611686018427387904ll;
constexpr int64_t kC5 = 3689348814741910323ll;
constexpr int64_t kC6 = 3074457345618258602ll;
constexpr int64_t kC7 = 2635249153387078802ll;
constexpr int64_t kC8 = 2305843009213693952ll;
constexpr int64_t kC9 = 2049638230412172402ll;

// nearest double to v 2^-F for 0 < v < 2^127 (F = 116 or 128)
EMT_LHD double fixed_to_double(u128 v, int F)
{
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    const int msb = hi ? 127 - clz64(hi) : 63 - clz64(lo);
    const int e = msb - F;  // unbiased exponent of the result
    uint64_t q;
    if (msb <= 52) {
        q = (uint64_t)v << (52 - msb);  // exact
    } else {
        const int sh = msb - 52;
        q = (uint64_t)(v >> sh);
        const u128 rest = v & (((u128)1 << sh) - 1), half = (u128)1 << (sh - 1);
        if (rest > half || (rest == half && (q & 1))) q += 1;  // nearest, ties to even
    }
    uint64_t b = ((uint64_t)(e + 1022) << 52) + q;  // q = 2^53 carries into the exponent
    double d;
    memcpy(&d, &b, 8);
    return d;
}

// ln x, rounded to nearest (see above)
EMT_LHD_CALL double log_rn(double x)
{
    uint64_t hx;
    memcpy(&hx, &x, 8);
    const int bexp = (int)(hx >> 52);  // sign bit included: negative x fails the test below
    if ((unsigned)(bexp - 1) >= 2046u) return log(x);
    const uint64_t M = (hx & ((1ull << 52) - 1)) | (1ull << 52);
    // X = M 2^-52 in [1, 1.5) or M 2^-53 in [0.75, 1)
    const int sh = M >= (3ull << 51) ? 1 : 0;
    const int E = bexp - 1023 + sh;
    const int j = (int)(M >> (44 + sh)) - 192;
#if defined(__CUDA_ARCH__)
    const uint64_t I = __ldg(&d_inv[j]);
    const i128 t = (i128)(((u128)__ldg(&d_thi[j]) << 64) | __ldg(&d_tlo[j]));
#else
    const uint64_t I = h_inv[j];
    const i128 t = (i128)(((u128)h_thi[j] << 64) | h_tlo[j]);
#endif
    // r 2^68 = M I 2^(1 - sh) - 2^68, at most 2^60 in magnitude: the low 64
    // bits of the product are the whole difference
    const int64_t R = (int64_t)((M * I) << (1 - sh));
    const int64_t r64 = R >> 4;  // r in Q0.64
    int64_t p = kC9;
    p = kC8 - mulhi(r64, p);
    p = kC7 - mulhi(r64, p);
    p = kC6 - mulhi(r64, p);
    p = kC5 - mulhi(r64, p);
    p = kC4 - mulhi(r64, p);
    p = kC3 - mulhi(r64, p);
    const i128 R2 = (i128)R * R;                      // r^2 2^136, exact
    const int64_t y = mulhi((int64_t)(R2 >> 58), p);  // r^2 P3 2^78 (r^2 <= 2^-16)
    // ln(1 + r) 2^128 = R 2^60 - R^2 2^-9 + R y 2^-18: relative error < 2^-77
    const i128 l1p = ((i128)R << 60) - (R2 >> 9) + (((i128)R * y) >> 18);
    // next to x = 1 the result is ln(1 + r) alone: rounded from 2^-128 units;
    // elsewhere |ln x| > 2^-8.1 and the sum is formed in 2^-116 units
    const bool central = E == 0 && t == 0;
    const i128 ln2 = (i128)(((u128)EMT_LN2_HI << 64) | EMT_LN2_LO);
    const i128 v = central ? l1p : ln2 * E + t + (l1p >> 12);
    if (v == 0) return 0.0;
    const double m = fixed_to_double(v < 0 ? (u128)(-v) : (u128)v, central ? 128 : 116);
    return v < 0 ? -m : m;
}

}  // namespace intlog
}  // namespace emt
