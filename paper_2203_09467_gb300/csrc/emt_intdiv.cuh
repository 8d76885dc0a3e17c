// emt_intdiv.cuh -- IEEE-754 binary64 division and square root on the
// integer pipe.
//
// GB300 executes FP64 at 2 fused multiply-adds per clock per SM (1/64 of
// its FP32 rate), while its integer units issue 64 operations per clock per
// SM.  A correctly rounded FP64 division built from FP64 multiply-adds
// (reciprocal estimate, Newton steps, remainder correction) occupies the
// narrow FP64 pipe for several instructions; the same quotient can be
// formed exactly from the operands' integer significands.  `div_rn(x, y)`
// returns bit for bit what `x / y` returns (round to nearest even): for
// normal operands with a normal quotient it divides the significands on
// the integer pipe; every other case (zeros, subnormals, infinities, NaNs,
// quotients near the ends of the exponent range) takes the native division.
//
// Method.  With x = A 2^ex, y = B 2^ey and A, B in [2^52, 2^53) (A doubled
// when A < B, so that A / B lies in [1, 2)), the result significand is
// RN(A 2^52 / B).  A quotient of two 53-bit integers is never a midpoint
// between two 53-bit integers (if A 2^53 = (2M + 1) B, the power of two in B
// would have to be at least 2^53), so RN(t) = (floor(2t) + 1) / 2 with
// 2t = A 2^53 / B, and only Q' = floor(A 2^53 / B) is needed:
//   1. R ~ 2^115 / B: an FP32 reciprocal of B's leading 24 bits (relative
//      error < 2^-22), then two Newton steps R += R (2^115 - B R) / 2^115 in
//      128-bit integer arithmetic (error ~ 2^-44, then within a few units of
//      the last place of the 64-bit R).
//   2. Q = floor(A R / 2^62): within one of Q' (A < 2^54, so a few units of
//      R move A R / 2^62 by less than 2^-7).
//   3. The exact remainder A 2^53 - Q B (|.| < 2^54, so its low 64 bits
//      are the whole value) corrects Q by one where needed.
//
// `sqrt_rn(x)` does the same for the square root: with x = N 2^(2k - 52),
// N in [2^52, 2^54), the result significand is RN(sqrt(N 2^52)), never a
// midpoint (its square would need more than 54 significant bits), so
// Q' = floor(sqrt(N 2^54)) suffices; Y ~ 2^63 / sqrt(N 2^-52) from an FP32
// reciprocal square root and two Newton steps Y += Y (1 - N Y^2 2^-178) / 2,
// Q = floor(N Y / 2^62) within one of Q', corrected by the exact remainder
// N 2^54 - Q^2 (|.| < 2^56).
//
// The FP32 reciprocal (square root) estimates are the only floating-point
// steps; their exact values do not matter, only their error bounds.  Host
// builds (the CPU test of this file) use correctly rounded FP32 results in
// their place, moved by up to three units of the last place to cover the
// hardware estimates' errors.
#pragma once

#include <stdint.h>
#include <math.h>
#include <string.h>

#if defined(__CUDACC__)
#define EMT_HD __host__ __device__ __forceinline__
// one out-of-line copy per kernel: the integer sequences are long, and
// inlined at every call site they overflowed the instruction cache of the
// step kernels (measured on GB300: the calorimeter 20% slower inlined)
#define EMT_HD_CALL static __host__ __device__ __noinline__
#else
#define EMT_HD static inline
#define EMT_HD_CALL static inline
#endif

namespace emt {
namespace intdiv {

typedef unsigned __int128 u128;
typedef __int128 i128;

EMT_HD uint64_t dbits(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}
EMT_HD double bitsd(uint64_t b)
{
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// FP32 reciprocal (or reciprocal square root) of b in [1, 4): relative
// error below 2^-22
template <bool kSqrt = false>
EMT_HD uint32_t rcp_f32_bits(float b)
{
#if defined(__CUDA_ARCH__)
    float r;
    if (kSqrt)
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    else
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
#else
    float r = kSqrt ? 1.0f / sqrtf(b) : 1.0f / b;
#endif
    uint32_t k;
    memcpy(&k, &r, 4);
#if defined(EMT_INTDIV_SEED_ERROR) && !defined(__CUDA_ARCH__)
    k += (uint32_t)EMT_INTDIV_SEED_ERROR(k);  // host test builds: a seed off by a few units
#endif
    return k;
}

// R ~ 2^115 / B for an integer significand B in [2^52, 2^53)
EMT_HD uint64_t recip115(uint64_t B)
{
    const uint32_t bb = 0x3F800000u | (uint32_t)((B >> 29) & 0x7FFFFFu);  // B's leading 24 bits, in [1, 2)
    float bf;
    memcpy(&bf, &bb, 4);
    const uint32_t rb = rcp_f32_bits(bf);                                  // in (1/2, 1]
    const uint64_t m = (uint64_t)((rb & 0x7FFFFFu) | 0x800000u);
    uint64_t R = m << (((rb >> 23) & 0xFFu) - 87u);                        // reciprocal * 2^63
    i128 D = ((i128)1 << 115) - (i128)((u128)B * R);                       // |D| < 2^94
    R += (uint64_t)(int64_t)(((i128)R * (int64_t)(D >> 51)) >> 64);
    D = ((i128)1 << 115) - (i128)((u128)B * R);                            // |D| < 2^72
    R += (uint64_t)(int64_t)(((i128)R * (int64_t)(D >> 12)) >> 103);
    return R;
}

// A divisor prepared once for several quotients (its reciprocal R).
struct Divisor {
    double y;
    uint64_t B, R;
    int ey;
};

EMT_HD Divisor divisor(double y)
{
    const uint64_t hy = dbits(y);
    Divisor d;
    d.y = y;
    d.ey = (int)((hy >> 52) & 0x7FF);
    d.B = (hy & ((1ull << 52) - 1)) | (1ull << 52);
    d.R = recip115(d.B);
    return d;
}

// x / d.y, correctly rounded (bit-identical to the IEEE division)
EMT_HD double div_rn(double x, const Divisor& d)
{
    const uint64_t hx = dbits(x);
    const int ex = (int)((hx >> 52) & 0x7FF);
    int er = ex - d.ey + 1023;
    // normal operands and a biased result exponent in [2, 2045] (so that
    // the halving of step 0 and the carry of the rounding stay normal)
    if ((unsigned)(ex - 1) >= 2046u || (unsigned)(d.ey - 1) >= 2046u || (unsigned)(er - 2) >= 2044u) return x / d.y;
    uint64_t A = (hx & ((1ull << 52) - 1)) | (1ull << 52);
    if (A < d.B) {
        A <<= 1;
        er -= 1;
    }
    uint64_t Q = (uint64_t)(((u128)A * d.R) >> 62);
    const int64_t rem = (int64_t)((A << 53) - Q * d.B);
    if (rem < 0) Q -= 1;
    else if (rem >= (int64_t)d.B) Q += 1;
    Q = (Q + 1) >> 1;  // in [2^52, 2^53]; 2^53 carries into the exponent below
    return bitsd(((hx ^ dbits(d.y)) & (1ull << 63)) | (((uint64_t)(er - 1) << 52) + Q));
}

// x / y, correctly rounded (bit-identical to the IEEE division)
EMT_HD_CALL double div_rn(double x, double y) { return div_rn(x, divisor(y)); }

// sqrt(x), correctly rounded (bit-identical to the IEEE square root)
EMT_HD_CALL double sqrt_rn(double x)
{
    const uint64_t hx = dbits(x);
    const int bexp = (int)(hx >> 52);  // sign bit included: negative x takes the native path
    if ((unsigned)(bexp - 1) >= 2046u) return sqrt(x);
    const int odd = (bexp - 1023) & 1;
    const uint64_t N = ((hx & ((1ull << 52) - 1)) | (1ull << 52)) << odd;  // in [2^52, 2^54)
    const int half_e = (bexp - 1023 - odd) / 2;
    // FP32 seed: N 2^-52 in [1, 4) from N's leading 24 bits
    const int top = (int)(N >> 53);  // 1 when N >= 2^53
    const uint32_t nb = ((uint32_t)(127 + top) << 23) | (uint32_t)((N >> (29 + top)) & 0x7FFFFFu);
    float nf;
    memcpy(&nf, &nb, 4);
    const uint32_t yb = rcp_f32_bits<true>(nf);  // in (1/2, 1]
    uint64_t Y = (uint64_t)((yb & 0x7FFFFFu) | 0x800000u) << (((yb >> 23) & 0xFFu) - 87u);  // y 2^63
    // Newton: y += y (1 - n y^2) / 2 with n y^2 = N (Y^2 2^-64) 2^-114
    i128 D = ((i128)1 << 114) - (i128)((u128)N * (uint64_t)(((u128)Y * Y) >> 64));  // |D| < 2^93
    Y += (uint64_t)(int64_t)(((i128)Y * (int64_t)(D >> 50)) >> 65);
    D = ((i128)1 << 114) - (i128)((u128)N * (uint64_t)(((u128)Y * Y) >> 64));       // |D| < 2^72
    Y += (uint64_t)(int64_t)(((i128)Y * (int64_t)(D >> 12)) >> 103);
    // floor(sqrt(N 2^54)) = floor(N y 2^-9) up to one
    uint64_t Q = (uint64_t)(((u128)N * Y) >> 62);
    const int64_t rem = (int64_t)((N << 54) - Q * Q);
    if (rem < 0) Q -= 1;
    else if (rem > (int64_t)(2 * Q)) Q += 1;
    Q = (Q + 1) >> 1;  // in [2^52, 2^53]
    return bitsd(((uint64_t)(half_e + 1022) << 52) + Q);
}

}  // namespace intdiv
}  // namespace emt
