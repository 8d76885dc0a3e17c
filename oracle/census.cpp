// census.cpp -- a count of the FP64 operations of the oracle's transport
// step, per operation kind (measurement infrastructure: it fixes the
// algorithmic FP64 work per track-step that the GPU step kernels' roofline
// is measured against, independently of how the kernels are compiled).
//
// The oracle's own source (emt_oracle.c) is compiled as C++ with every
// `double` replaced by F64, a value type that performs the same IEEE
// operation and counts it while counting is on.  Nothing in the oracle's
// arithmetic changes; the counts are of the operations the definition of
// the method performs (the oracle's operation order), not of any GPU code.
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

namespace census {
enum Kind { kAdd, kSub, kMul, kDiv, kFma, kSqrt, kCmp, kNeg, kMinMax, kRound, kCbrt, kLog, kExp, kLog1p, kExpm1,
            kSin, kCos, kPow, kKinds };
static unsigned long long count[kKinds];
static int on = 0;
static inline void tick(Kind k)
{
    if (on) ++count[k];
}
}  // namespace census

struct F64 {
    double v;
    F64() = default;
    constexpr F64(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    explicit operator unsigned() const { return (unsigned)v; }
    explicit operator long() const { return (long)v; }
    explicit operator unsigned long() const { return (unsigned long)v; }
    explicit operator long long() const { return (long long)v; }
    explicit operator unsigned long long() const { return (unsigned long long)v; }
    F64& operator+=(F64 o);
    F64& operator-=(F64 o);
    F64& operator*=(F64 o);
    F64& operator/=(F64 o);
};

static inline double val(F64 x) { return x.v; }
static inline double val(double x) { return x; }

#define CENSUS_BIN(OP, KIND)                                                             \
    static inline F64 operator OP(F64 a, F64 b)                                          \
    {                                                                                    \
        census::tick(census::KIND);                                                      \
        return F64(a.v OP b.v);                                                          \
    }                                                                                    \
    static inline F64 operator OP(F64 a, double b)                                       \
    {                                                                                    \
        census::tick(census::KIND);                                                      \
        return F64(a.v OP b);                                                            \
    }                                                                                    \
    static inline F64 operator OP(double a, F64 b)                                       \
    {                                                                                    \
        census::tick(census::KIND);                                                      \
        return F64(a OP b.v);                                                            \
    }
CENSUS_BIN(+, kAdd)
CENSUS_BIN(-, kSub)
CENSUS_BIN(*, kMul)
CENSUS_BIN(/, kDiv)
#undef CENSUS_BIN

#define CENSUS_CMP(OP)                                                                   \
    static inline bool operator OP(F64 a, F64 b)                                         \
    {                                                                                    \
        census::tick(census::kCmp);                                                      \
        return a.v OP b.v;                                                               \
    }                                                                                    \
    static inline bool operator OP(F64 a, double b)                                      \
    {                                                                                    \
        census::tick(census::kCmp);                                                      \
        return a.v OP b;                                                                 \
    }                                                                                    \
    static inline bool operator OP(double a, F64 b)                                      \
    {                                                                                    \
        census::tick(census::kCmp);                                                      \
        return a OP b.v;                                                                 \
    }
CENSUS_CMP(<)
CENSUS_CMP(>)
CENSUS_CMP(<=)
CENSUS_CMP(>=)
CENSUS_CMP(==)
CENSUS_CMP(!=)
#undef CENSUS_CMP

inline F64& F64::operator+=(F64 o) { return *this = *this + o; }
inline F64& F64::operator-=(F64 o) { return *this = *this - o; }
inline F64& F64::operator*=(F64 o) { return *this = *this * o; }
inline F64& F64::operator/=(F64 o) { return *this = *this / o; }
static inline F64 operator-(F64 a)
{
    census::tick(census::kNeg);
    return F64(-a.v);
}
static inline F64 operator+(F64 a) { return a; }

#define CENSUS_F1(NAME, KIND)                    \
    static inline F64 NAME(F64 x)                \
    {                                            \
        census::tick(census::KIND);              \
        return F64(::NAME(x.v));                 \
    }
CENSUS_F1(sqrt, kSqrt)
CENSUS_F1(cbrt, kCbrt)
CENSUS_F1(log, kLog)
CENSUS_F1(log10, kLog)
CENSUS_F1(exp, kExp)
CENSUS_F1(log1p, kLog1p)
CENSUS_F1(expm1, kExpm1)
CENSUS_F1(sin, kSin)
CENSUS_F1(cos, kCos)
CENSUS_F1(floor, kRound)
CENSUS_F1(ceil, kRound)
#undef CENSUS_F1
static inline F64 fabs(F64 x) { return F64(::fabs(x.v)); }  // a sign-bit operation
template <class A, class B>
static inline F64 fmax(A a, B b)
{
    census::tick(census::kMinMax);
    return F64(::fmax(val(a), val(b)));
}
template <class A, class B>
static inline F64 pow(A a, B b)
{
    census::tick(census::kPow);
    return F64(::pow(val(a), val(b)));
}
template <class A, class B, class C>
static inline F64 fma(A a, B b, C c)
{
    census::tick(census::kFma);
    return F64(::fma(val(a), val(b), val(c)));
}

#define double F64
#include "emt_oracle.c"
#undef double

extern "C" {
// counting on (1) or off (0); reset clears the counts; read copies them
// in the order of census::Kind
void orc_census_enable(int enable) { census::on = enable; }
void orc_census_reset(void) { memset(census::count, 0, sizeof census::count); }
int orc_census_read(unsigned long long* out, int cap)
{
    const int n = cap < census::kKinds ? cap : census::kKinds;
    for (int k = 0; k < n; ++k) out[k] = census::count[k];
    return census::kKinds;
}
}
