// emt_device.cuh -- device-side data layout, random streams, table
// lookups, navigation, field propagation and interaction samplers of the
// EM transport step (arXiv:2203.09467, Secs. 2.1-2.3).
//
// Templated on the physics real type R: double for the FP64 path (built
// with --fmad=false so every expression rounds exactly as written) and
// float for the mixed path (positions, boundary distances and tallies stay
// FP64).  Each formula cites the textbook closed form it evaluates; the
// operation order of the FP64 instantiation is the library's definition of
// the method and is what the FP64 tests compare against.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "emt_intdiv.cuh"
#include "emt_intlog.cuh"

namespace emt {

constexpr double kMe = 0.51099895;          // electron mass, MeV (CODATA 2018)
constexpr double kRe = 2.8179403262e-13;    // classical electron radius, cm
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kNa = 6.02214076e23;       // 1/mol
constexpr double kPi = 3.14159265358979323846;
constexpr double kFieldC = 2.99792458;      // curvature per (T / MeV), 1/cm
constexpr int kMaxMat = 16;
constexpr int kMaxLayers = 4096;
constexpr int kVolWorld = -1;               // vacuum of the world box
constexpr int kVolOut = -2;                 // left the world
constexpr int kGeomLayers = 0;              // slabs stacked along z in a world box
constexpr int kGeomCylinders = 1;           // concentric shells about the z axis
constexpr int kNq = 4;                      // table quantities per node
// Rejection loops accept their candidate after kMaxTrials trials: a bound
// against non-finite input (every acceptance probability is >= 1/3).
constexpr int kMaxTrials = 1000;

// status bits written by kernels (host reads after each run)
// track selection (active budget per step)
constexpr int kSelectOrder = 0;      // the first max_active tracks of the input order
constexpr int kSelectLowEnergy = 1;  // the max_active tracks of lowest energy
constexpr int kEBins = 128;          // energy classes: quarter octaves from 2^-16 MeV
constexpr int kEBase = 112 << 2;     // (FP32 exponent << 2 | two mantissa bits) of class 0
// physics options (process-mask bits beyond the six discrete processes)
constexpr unsigned kProcMsc = 64u;      // multiple scattering of e+-
constexpr unsigned kProcAngular = 128u;  // angles of brems photons, pair leptons, photoelectrons
constexpr unsigned kProcRayleigh = 256u;  // Rayleigh scattering of photons
constexpr double kBohr = 0.529177210903e-8;  // Bohr radius, cm (CODATA 2018)
constexpr double kHbarC = 197.3269804e-13;   // hbar c, MeV cm (CODATA 2018)
constexpr uint32_t kMscDraw = 1u << 20;  // draw index of the two msc uniforms of a step
constexpr int kStatusQueueOverflow = 1;
constexpr int kStatusBadTrack = 2;
constexpr int kStatusTimeout = 4;  // a bounded device wait gave up (persistent step loop)

// ------------------------------------------------------------------ math
// FP64 logarithm on the integer pipe (emt_intlog.cuh), FP32 native
__device__ __forceinline__ double mlog(double x) { return intlog::log_rn(x); }
__device__ __forceinline__ float mlog(float x) { return logf(x); }
__device__ __forceinline__ double mexp(double x) { return exp(x); }
__device__ __forceinline__ float mexp(float x) { return expf(x); }
// a * b + c with one rounding (the interpolations and the straight move,
// as in the oracle)
__device__ __forceinline__ double mfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float mexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double mlog1p(double x) { return log1p(x); }
__device__ __forceinline__ float mlog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double msqrt(double x) { return intdiv::sqrt_rn(x); }  // integer pipe, exact
__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double msin(double x) { return sin(x); }
__device__ __forceinline__ float msin(float x) { return sinf(x); }
__device__ __forceinline__ double mcos(double x) { return cos(x); }
__device__ __forceinline__ float mcos(float x) { return cosf(x); }
__device__ __forceinline__ double mfmax(double a, double b) { return fmax(a, b); }
// a / b: FP64 quotients on the integer pipe (bit-identical to the IEEE
// division; GB300's FP64 pipe is its narrowest), FP32 quotients native
__device__ __forceinline__ double mdiv(double a, double b) { return intdiv::div_rn(a, b); }
__device__ __forceinline__ float mdiv(float a, float b) { return a / b; }
// a quotient whose divisor several numerators share
struct DivisorF {
    float y;
};
__device__ __forceinline__ intdiv::Divisor mdivisor(double y) { return intdiv::divisor(y); }
__device__ __forceinline__ DivisorF mdivisor(float y) { return DivisorF{y}; }
__device__ __forceinline__ double mdiv(double a, const intdiv::Divisor& d) { return intdiv::div_rn(a, d); }
__device__ __forceinline__ float mdiv(float a, const DivisorF& d) { return a / d.y; }
__device__ __forceinline__ float mfmax(float a, float b) { return fmaxf(a, b); }

// ------------------------------------------------------------------ conversions
// Measured on GB300: exact conversions between the physics type and FP64
// are fastest as the hardware instructions, but an FP32 estimate of a
// double (bin search, navigation prefilter) is cheaper from integer
// operations on the bit pattern than from a rounding conversion.

// double -> float truncated toward zero, for estimates only (relative error
// < 2^-23; magnitudes below the float range give 0, above it infinity)
__device__ __forceinline__ float d2f_est(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// the physics type R to and from FP64 (identity for the FP64 path)
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
template <typename R>
__device__ __forceinline__ R from_d(double x);
template <>
__device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
__device__ __forceinline__ float est_f(double x) { return d2f_est(x); }
__device__ __forceinline__ float est_f(float x) { return x; }

// ------------------------------------------------------------------ layout
// One ping-pong side of the track store, structure of arrays.  Photons
// occupy [0, nG) from the front, charged tracks [Q-nC, Q) from the back.
template <typename R>
struct Tracks {
    double* x;
    double* y;
    double* z;
    R* ux;
    R* uy;
    R* uz;
    R* T;
    uint64_t* uid;
    uint32_t* ev;    // event slot
    uint32_t* step;  // steps taken by this track
    uint32_t* tv;    // type (bits 0-7) | (volume + 2) << 8
};

// scheduling classes of charged tracks in a field: class 0 holds the most
// expensive tracks (an estimated 72 or more RK4 substeps), classes 1-7 hold
// ranges of 2 to 16 substep counts, and classes 8-27 hold a single count
// each, 20 down to 1, where most tracks of a calorimeter lie
constexpr int kSortKeys = 32;
__host__ __device__ constexpr int substep_class(int n)
{
    return n <= 20   ? 28 - n
           : n <= 22 ? 7
           : n <= 25 ? 6
           : n <= 29 ? 5
           : n <= 35 ? 4
           : n <= 43 ? 3
           : n <= 55 ? 2
           : n <= 71 ? 1
                     : 0;
}

// state of the grid barrier of the persistent step loop (zeroed before
// each launch)
struct GridSync {
    unsigned count;  // blocks arrived at the current barrier
    unsigned gen;    // barriers completed
    unsigned iters;  // steps run by the launch
    unsigned pad;
};

// per-iteration counters, rotating over three slots (input, output, clear)
struct Counters {
    int n[2];      // photons, charged
    int work;      // chunk dispenser
    int used;      // growth tokens taken (steps with two outputs)
    int n_int;     // split schedule: tracks queued for an interaction
    int work_b;    // split schedule: chunk dispenser of the interaction kernel
    int ticket;    // track selection: tickets of the boundary energy class
    int spilled;   // host spill: tracks written to the spill buffer
    int kbin[kSortKeys];  // field: charged input tracks per scheduling class
    int kcur[kSortKeys];  // field: places taken per class while the order is written
};

// Split schedule: tracks that interact in a step, queued by the transport
// kernel for the interaction kernel (structure of arrays, Q entries).
template <typename R>
struct InterQueue {
    double* x;
    double* y;
    double* z;
    R* ux;
    R* uy;
    R* uz;
    R* T;
    uint64_t* uid;
    double* dep;     // energy deposited by the transport part of the step
    uint32_t* ev;
    uint32_t* step;
    uint32_t* tv;    // type | (volume + 2) << 8 | model << 24
    uint32_t* src;   // index of the track in the input buffer (for deferral)
};

template <typename R>
struct Params {
    // tables: tab[((m * 3 + p) * n_grid + node) * 4 + q]
    const R* grid;
    const R* tab;
    const R* igrid;  // 1 / (grid[n+1] - grid[n])
    const R* irs;    // [(m * 3 + p) * n_grid + n]: 1 / (R[n+1] - R[n]) of the range tables
    const R* dgrid;  // grid[n+1] - grid[n]
    const R* dtab;   // layout of tab: tab[n+1][q] - tab[n][q]
    int n_grid;
    int bpd;
    float log10_lo;  // log10(grid[0]) for the bin guess
    const double* bk;
    const int* vacuum;
    const double* x0;     // radiation length per material (cm)
    const double* ray_a;  // Rayleigh screening radius per material (cm)
    unsigned mask;     // process mask (physics options: kProcMsc, kProcAngular)
    double cut[3];
    double step_frac, final_range;
    float cutf[3];  // the same in FP32 (mixed path)
    float step_fracf, final_rangef;
    // geometry: layers (zb = plane positions) or cylinders (zb = shell
    // radii, zb[0] = 0, the stack spans |z| <= half_z)
    int geom;
    double half_z;
    const double* zb;
    const int* lmat;
    const int* lbin;
    int n_layers;
    double hx, hy;
    // ord_key of the lateral bounds of a layer's chord test, formed once
    // when the geometry is loaded: -hx + m, hx - m, -hy + m, hy - m
    // (m = kChordMargin)
    long long kxy[4];
    double wlo[3], whi[3];
    double B[3];
    double bmag;
    double rk_delta, max_field_step;
    int has_field;
    int max_steps;
    // scoring
    double* hist;  // [slot][hstride]; column n_bins collects unbinned deposits
    int hstride;
    int n_bins;
    int score_z;           // bins along z: floor((z - zs_lo) * zs_scale); else per volume
    double zs_lo, zs_scale;
    unsigned long long* step_hist;  // [3][step_bins] steps per finished track, or null
    int step_bins;
    double* ledger;                 // [slot][3] escaped, killed, e_in
    unsigned long long* counts;     // [slot][2] steps, tracks
    const uint64_t* event_id;       // [slot]
    int* live;                      // [slot] tracks alive (+1 submission token)
    unsigned* done_ring;            // [max_events] slots of finished events
    unsigned* done_head;            // total finished events (ring index)
    unsigned long long* total_steps;  // [0] track-steps taken, [1] deferred copies, [2] held copies,
                                      // [3] RK4 substeps
    int max_events;
    uint32_t seed;
    // queues
    Tracks<R> q[2];
    long long Q;
    Counters* cnt;  // [3]
    int* status;
    InterQueue<R> iq;      // split and pipelined schedules
    InterQueue<R> iq_alt;  // pipelined schedule: the second queue (iterations alternate)
    // split schedule in a field: scheduling class of each charged input
    // track (skey[i], i = index in the charged region) and the order in
    // which the transport kernel takes them (sperm: indices, most
    // expensive class first); Q entries each
    uint8_t* skey;
    uint32_t* sperm;
    // track selection: at most max_active tracks step per iteration (0 =
    // all), chosen by select_policy; the others are held (copied
    // unchanged).  ehist[3][kEBins]: energy classes of each counter slot's
    // tracks (rotating with the counters).
    long long max_active;
    int select_policy;
    unsigned* ehist;
    // host spill: held tracks beyond the spill_above lowest-energy ones are
    // written to the spill buffer (spill_cap records) instead of the output,
    // and the host moves them to its memory (0 = off)
    long long spill_above;
    Tracks<R> spill;
    long long spill_cap;
    int* spill_ticket;  // tickets of the spill boundary class, [3] rotating
};

// energy class of a kinetic energy (monotonic in T): the FP32 exponent and
// two leading mantissa bits, offset and clamped to [0, kEBins)
__device__ __forceinline__ int energy_class(float T)
{
    const int c = (int)(__float_as_uint(T) >> 21) - kEBase;
    return c < 0 ? 0 : (c >= kEBins ? kEBins - 1 : c);
}

// production cut of particle type t and the e+- step-limit constants in R
template <typename R>
__device__ __forceinline__ R pcut(const Params<R>& p, int t)
{
    if constexpr (sizeof(R) == 8)
        return p.cut[t];
    else
        return p.cutf[t];
}
template <typename R>
__device__ __forceinline__ R pstep_frac(const Params<R>& p)
{
    if constexpr (sizeof(R) == 8)
        return p.step_frac;
    else
        return p.step_fracf;
}
template <typename R>
__device__ __forceinline__ R pfinal_range(const Params<R>& p)
{
    if constexpr (sizeof(R) == 8)
        return p.final_range;
    else
        return p.final_rangef;
}

__device__ __forceinline__ uint32_t pack_tv(int type, int vol) { return (uint32_t)type | ((uint32_t)(vol + 2) << 8); }
__device__ __forceinline__ int tv_type(uint32_t tv) { return (int)(tv & 0xFFu); }
__device__ __forceinline__ int tv_vol(uint32_t tv) { return (int)(tv >> 8) - 2; }

// ------------------------------------------------------------------ RNG
// Philox4x32-10 (Salmon et al., SC'11): multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85, 10 rounds.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c[0];
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Draw stream of one track step: key (lo32(event), hi32(event) ^ seed),
// counter (lo32(uid), hi32(uid), step, block).  FP64: draw j uses block
// j >> 1, words 2(j&1) (low half) and 2(j&1)+1 (high half) as a 64-bit
// word w; u = (floor(w / 2^12) + 1/2) 2^-52, formed exactly as
// (1 + m 2^-52) - (1 - 2^-53).  FP32: draw j uses block j >> 2, word j & 3,
// u = (floor(w / 2^9) + 1/2) 2^-23.
struct Draws {
    uint32_t k0, k1, c0, c1, step;
    uint32_t next;
    uint32_t blk;
    uint32_t w[4];

    __device__ __forceinline__ void init(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t s)
    {
        k0 = (uint32_t)event_id;
        k1 = (uint32_t)(event_id >> 32) ^ seed;
        c0 = (uint32_t)uid;
        c1 = (uint32_t)(uid >> 32);
        step = s;
        next = 0;
        blk = 0xFFFFFFFFu;
    }
    __device__ __forceinline__ void fill(uint32_t b)
    {
        if (b != blk) {
            w[0] = c0;
            w[1] = c1;
            w[2] = step;
            w[3] = b;
            philox10(w, k0, k1);
            blk = b;
        }
    }
    __device__ __forceinline__ double u64(uint32_t j)
    {
        fill(j >> 1);
        uint32_t lo = (j & 1u) ? w[2] : w[0];
        uint32_t hi = (j & 1u) ? w[3] : w[1];
        uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 12;
        return __longlong_as_double((long long)(0x3FF0000000000000ull | m)) - (1.0 - 0x1p-53);
    }
    __device__ __forceinline__ float u32(uint32_t j)
    {
        fill(j >> 2);
        // a select chain keeps the words in registers (an indexed read
        // would place w in local memory)
        const uint32_t v = (j & 2u) ? ((j & 1u) ? w[3] : w[2]) : ((j & 1u) ? w[1] : w[0]);
        return __int_as_float((int)(0x3F800000u | (v >> 9))) - (1.0f - 0x1p-24f);
    }
};

template <typename R>
struct DrawOf;
template <>
struct DrawOf<double> {
    static __device__ __forceinline__ double at(Draws& d, uint32_t j) { return d.u64(j); }
};
template <>
struct DrawOf<float> {
    static __device__ __forceinline__ float at(Draws& d, uint32_t j) { return d.u32(j); }
};

template <typename R>
__device__ __forceinline__ R draw(Draws& d)
{
    R u = DrawOf<R>::at(d, d.next);
    d.next += 1;
    return u;
}

// child k of (uid, step): key word 0 ^ 0x5EC0DA7A, counter word 3 = 2^31 + k
__device__ __forceinline__ uint64_t child_uid(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step,
                                              uint32_t k)
{
    uint32_t c[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), step, 0x80000000u + k};
    philox10(c, (uint32_t)event_id ^ 0x5EC0DA7Au, (uint32_t)(event_id >> 32) ^ seed);
    return ((uint64_t)c[1] << 32) | (uint64_t)c[0];
}

// ------------------------------------------------------------------ tables
// Comparisons on the integer pipe (the FP64 pipe is narrow).  The signed
// order of the bit patterns of two IEEE values is their numeric order when
// neither is NaN and at least one of them is > 0: two non-negative values
// order like their bits, and a negative value or -0 has a negative pattern,
// below every positive one.  Every call site has one operand > 0 (a grid
// node, a cut, a step limit, a range, a cross-section sum).
__device__ __forceinline__ bool le_pos(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
__device__ __forceinline__ bool le_pos(float a, float b) { return __float_as_int(a) <= __float_as_int(b); }
__device__ __forceinline__ bool lt_pos(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool lt_pos(float a, float b) { return a < b; }
// a > 0 and a != 0, exact for every value (NaN: false and true)
__device__ __forceinline__ bool gt_zero(double a) { return __double_as_longlong(a) > 0; }
__device__ __forceinline__ bool gt_zero(float a) { return a > 0.0f; }
__device__ __forceinline__ bool nonzero(double a) { return ((unsigned long long)__double_as_longlong(a) << 1) != 0ull; }
// An integer key whose signed order is the numeric order of any two
// non-NaN doubles of either sign: the magnitude bits, negated for a
// negative value (so -0 and +0 both map to 0).  A NaN maps beyond every
// finite value on its sign's side.
__host__ __device__ __forceinline__ long long ord_key(double a)
{
#ifdef __CUDA_ARCH__
    const long long b = __double_as_longlong(a);
#else
    long long b;
    memcpy(&b, &a, sizeof b);
#endif
    const long long m = b & 0x7fffffffffffffffll;
    return b < 0 ? -m : m;
}

// node n with grid[n] <= E < grid[n+1], clamped to [0, n_grid-2]: an FP32
// logarithm guesses, exact comparisons with the nodes decide.
template <typename R>
__device__ __forceinline__ int find_bin(const Params<R>& p, R E)
{
    float g = ((float)p.bpd) * (log10f(est_f(E)) - p.log10_lo);
    int n = (int)g;
    int top = p.n_grid - 2;
    n = n < 0 ? 0 : (n > top ? top : n);
    while (n > 0 && !le_pos(p.grid[n], E)) --n;
    while (n < top && le_pos(p.grid[n + 1], E)) ++n;
    return n;
}

// piecewise-linear in E between nodes, constant outside the grid
template <typename R>
struct Lookup {
    int n;
    R f;
    int clamp;  // -1 below grid, +1 above, 0 inside
};

template <typename R>
__device__ __forceinline__ Lookup<R> locate_energy(const Params<R>& p, R E)
{
    Lookup<R> l;
    l.clamp = 0;
    if (le_pos(E, p.grid[0])) {
        l.clamp = -1;
        l.n = 0;
        l.f = R(0);
        return l;
    }
    if (le_pos(p.grid[p.n_grid - 1], E)) {
        l.clamp = 1;
        l.n = p.n_grid - 2;
        l.f = R(0);
        return l;
    }
    l.n = find_bin(p, E);
    l.f = (E - p.grid[l.n]) * p.igrid[l.n];  // the reciprocal width, rounded once
    return l;
}

// t, dt: the rows of tab and dtab of one material and particle type
template <typename R>
__device__ __forceinline__ R xs_value(const Params<R>& p, const R* t, const R* dt, const Lookup<R>& l, int q)
{
    if (l.clamp < 0) return t[q];
    if (l.clamp > 0) return t[(p.n_grid - 1) * kNq + q];
    return mfma(dt[l.n * kNq + q], l.f, t[l.n * kNq + q]);
}

// range: linear through the origin below the grid, linear between nodes,
// extrapolated with the last slope above
template <typename R>
__device__ __forceinline__ R range_value(const Params<R>& p, const R* t, const R* dt, R T, const Lookup<R>& l)
{
    if (lt_pos(T, p.grid[0])) return t[3] * mdiv(T, p.grid[0]);
    int n = l.n;
    R f = l.f;
    if (l.clamp > 0) f = (T - p.grid[n]) * p.igrid[n];
    return mfma(dt[n * kNq + 3], f, t[n * kNq + 3]);
}

// inverse of range_value with the range intervals' reciprocal widths irs;
// nstart = bin of the pre-step energy (the answer lies at or below it
// because r <= R(T))
template <typename R>
__device__ __forceinline__ R inv_range(const Params<R>& p, const R* t, const R* irs, R r, int nstart)
{
    if (lt_pos(r, t[3])) return p.grid[0] * mdiv(r, t[3]);
    int n = nstart;
    while (n > 0 && !le_pos(t[n * kNq + 3], r)) --n;
    int top = p.n_grid - 2;
    while (n < top && le_pos(t[(n + 1) * kNq + 3], r)) ++n;
    R f = (r - t[n * kNq + 3]) * irs[n];
    return mfma(p.dgrid[n], f, p.grid[n]);
}

// ------------------------------------------------------------------ geometry
struct Exit {
    double t;
    double plane;
    int next;
    int axis;
};

// layer containing z for entries through a side face: largest j with
// zb[j] <= z, clamped to [0, L-1]
__device__ __forceinline__ int layer_at(const double* zb, int L, double z)
{
    int lo = 0, hi = L - 1;  // answer in [lo, hi]
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (zb[mid] <= z)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Cylinders: exit parameter t >= 0 along d (any length) from x in shell
// vol.  Candidates in the order end plane, outer surface, inner surface;
// the smallest wins, ties to the earlier.  The surface rho = r meets
// x + t d where a t^2 + 2 b t + c = 0 (a = dx^2 + dy^2, b = x dx + y dy,
// c = x^2 + y^2 - r^2).  Outer surface: the larger root, in the form free
// of cancellation for the sign of b; inner surface: only moving inward
// (b < 0) with a non-negative discriminant, the smaller root.  A radial
// crossing moves to the neighbouring shell; the end planes and the
// outermost surface lead out of the world (no snapping onto a curved
// surface: the volume index is exact, the position is the computed one).
template <typename R>
__device__ __forceinline__ Exit nav_exit_cyl(const Params<R>& p, int vol, const double x[3], const double d[3])
{
    Exit e;
    e.t = __longlong_as_double(0x7FF0000000000000ll);
    e.next = kVolOut;
    e.axis = -1;
    e.plane = 0.0;
    if (d[2] != 0.0) {
        const double pl = d[2] > 0.0 ? p.half_z : -p.half_z;
        e.t = mdiv(pl - x[2], d[2]);
        e.axis = 2;
        e.plane = pl;
    }
    const double a = d[0] * d[0] + d[1] * d[1];
    if (a > 0.0) {
        const double b = x[0] * d[0] + x[1] * d[1];
        const double q = x[0] * x[0] + x[1] * x[1];
        const double ro = p.zb[vol + 1];
        const double c = q - ro * ro;
        double disc = b * b - a * c;
        if (disc < 0.0) disc = 0.0;
        const double sq = msqrt(disc);
        const double t = b > 0.0 ? mdiv(-c, b + sq) : mdiv(sq - b, a);
        if (t < e.t) {
            e.t = t;
            e.axis = -1;
            e.plane = 0.0;
            e.next = vol + 1 < p.n_layers ? vol + 1 : kVolOut;
        }
        if (vol > 0 && b < 0.0) {
            const double ri = p.zb[vol];
            const double ci = q - ri * ri;
            const double di = b * b - a * ci;
            if (di >= 0.0) {
                const double ti = mdiv(ci, msqrt(di) - b);
                if (ti < e.t) {
                    e.t = ti;
                    e.axis = -1;
                    e.plane = 0.0;
                    e.next = vol - 1;
                }
            }
        }
    }
    if (e.t < 0.0) e.t = 0.0;
    return e;
}

// logical volume of a starting point (primaries): the layer (or shell)
// containing it, the world vacuum, or kVolOut
template <typename R>
__device__ __forceinline__ int locate_volume(const Params<R>& p, const double x[3])
{
    if (p.geom == kGeomCylinders) {
        const double q = x[0] * x[0] + x[1] * x[1];
        const double rmax = p.zb[p.n_layers];
        if (!(x[2] >= -p.half_z && x[2] <= p.half_z) || !(q < rmax * rmax)) return kVolOut;
        int lo = 0, hi = p.n_layers - 1;  // largest j with zb[j]^2 <= q
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.zb[mid] * p.zb[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    if (x[0] >= -p.hx && x[0] <= p.hx && x[1] >= -p.hy && x[1] <= p.hy && x[2] >= p.zb[0] &&
        x[2] <= p.zb[p.n_layers])
        return layer_at(p.zb, p.n_layers, x[2]);
    if (x[0] < p.wlo[0] || x[0] > p.whi[0] || x[1] < p.wlo[1] || x[1] > p.whi[1] || x[2] < p.wlo[2] ||
        x[2] > p.whi[2])
        return kVolOut;
    return kVolWorld;
}

// histogram column of a deposit in volume vol at height z (column n_bins
// collects deposits outside every bin)
template <typename R>
__device__ __forceinline__ int score_col(const Params<R>& p, int vol, double z)
{
    if (p.score_z) {
        const double f = floor((z - p.zs_lo) * p.zs_scale);
        return (f >= 0.0 && f < (double)p.n_bins) ? (int)f : p.n_bins;
    }
    if (vol >= 0) {
        const int b = p.lbin[vol];
        if (b >= 0 && b < p.n_bins) return b;
    }
    return p.n_bins;
}

// exit parameter t >= 0 along d (any length) from point x in volume vol.
// Layer: z plane first, then the x and y walls; ties keep the earlier.
// World vacuum: stack faces (z, x, y) first, then the world walls.
template <typename R>
__device__ __forceinline__ Exit nav_exit_layers(const Params<R>& p, int vol, const double x[3], const double d[3])
{
    Exit e;
    e.t = __longlong_as_double(0x7FF0000000000000ll);
    e.next = kVolOut;
    e.axis = -1;
    e.plane = 0.0;
    if (vol >= 0) {
        // Candidates: the z plane ahead, then the x and y walls ahead; the
        // exit is the smallest (pl - x)/d, ties to the earlier candidate.
        // FP32 estimates of the three quotients (operands truncated to FP32
        // by integer operations, quotient relative error < 1e-6)
        // select the candidates that can be the minimum (within 1e-5 of the
        // smallest estimate); only those are divided in FP64, in the same
        // order and with the same strict comparison, so the result is the
        // one all three FP64 divisions would give.  An estimate is trusted
        // only where its divisor is in the FP32 normal range: a nonzero
        // direction component below it truncates to 0 and its estimate
        // (infinite, or 0/0 from a point exactly on the wall) says nothing,
        // so that candidate is always divided.  The numerator (a distance
        // within the geometry) cannot overflow the FP32 range.
        const int L = p.n_layers;
        double pl[3], diff[3];
        int nx[3];
        bool has[3];
        float tf[3];
        bool sure[3];
        has[2] = nonzero(d[2]);
        if (gt_zero(d[2])) {
            pl[2] = p.zb[vol + 1];
            nx[2] = vol + 1 < L ? vol + 1 : kVolWorld;
        } else {
            pl[2] = p.zb[vol];
            nx[2] = vol > 0 ? vol - 1 : kVolWorld;
        }
        has[0] = nonzero(d[0]);
        pl[0] = gt_zero(d[0]) ? p.hx : -p.hx;
        nx[0] = kVolWorld;
        has[1] = nonzero(d[1]);
        pl[1] = gt_zero(d[1]) ? p.hy : -p.hy;
        nx[1] = kVolWorld;
        float tmin = __int_as_float(0x7F800000);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!has[a]) continue;
            diff[a] = pl[a] - x[a];
            const float df = d2f_est(d[a]);
            sure[a] = df != 0.0f;
            tf[a] = d2f_est(diff[a]) / df;
            tmin = fminf(tmin, tf[a]);
        }
        // a non-finite smallest estimate (a direction component below the
        // FP32 range) falls back to dividing every candidate
        const float thr = (tmin > -1e30f && tmin < 1e30f) ? tmin + fabsf(tmin) * 1e-5f + 1e-30f
                                                          : __int_as_float(0x7F800000);
        const int order[3] = {2, 0, 1};
#pragma unroll
        for (int oi = 0; oi < 3; ++oi) {
            const int a = order[oi];
            if (!has[a] || (sure[a] && !(tf[a] <= thr))) continue;
            double t = mdiv(diff[a], d[a]);
            if (t < e.t) {
                e.t = t;
                e.next = nx[a];
                e.axis = a;
                e.plane = pl[a];
            }
        }
    } else {
        const double lo[3] = {-p.hx, -p.hy, p.zb[0]};
        const double hi[3] = {p.hx, p.hy, p.zb[p.n_layers]};
        const int order[3] = {2, 0, 1};
#pragma unroll
        for (int oi = 0; oi < 3; ++oi) {
            int a = order[oi];
            if (d[a] == 0.0) continue;
            double pl = d[a] > 0.0 ? lo[a] : hi[a];
            double t = mdiv(pl - x[a], d[a]);
            if (!(t >= 0.0) || !(t < e.t)) continue;
            bool ok = true;
            double qz = 0.0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                double qb = x[b] + t * d[b];
                if (qb < lo[b] || qb > hi[b]) ok = false;
                if (b == 2) qz = qb;
            }
            if (!ok) continue;
            e.t = t;
            e.axis = a;
            e.plane = pl;
            if (a == 2)
                e.next = d[2] > 0.0 ? 0 : p.n_layers - 1;
            else
                e.next = layer_at(p.zb, p.n_layers, qz);
        }
#pragma unroll
        for (int oi = 0; oi < 3; ++oi) {
            int a = order[oi];
            if (d[a] == 0.0) continue;
            double pl = d[a] > 0.0 ? p.whi[a] : p.wlo[a];
            double t = mdiv(pl - x[a], d[a]);
            if (t < e.t) {
                e.t = t;
                e.next = kVolOut;
                e.axis = a;
                e.plane = pl;
            }
        }
    }
    if (e.t < 0.0) e.t = 0.0;
    return e;
}

// the exit of geometry kind G (kernels are instantiated per kind)
template <int G, typename R>
__device__ __forceinline__ Exit nav_exit(const Params<R>& p, int vol, const double x[3], const double d[3])
{
    if constexpr (G == kGeomCylinders)
        return nav_exit_cyl(p, vol, x, d);
    else
        return nav_exit_layers(p, vol, x, d);
}

// ------------------------------------------------------------------ field
// classical RK4 in path length on (x, u), du/ds = kq u x B, |p| fixed
// during the step; u renormalised after each substep.  The direction and
// its derivatives are evaluated in R (FP64 path: double, in the operation
// order of the definition; mixed path: float), positions accumulate in FP64.
template <typename R>
__device__ __forceinline__ void rk4(const Params<R>& p, R kq, const double x[3], const R u[3], R hs, R h6,
                                    double xo[3], R uo[3])
{
    // h6 = hs / 6, rounded once by the caller (the same quotient for every
    // substep of one length)
    // products added to a sum are fused (one rounding each), as in the oracle
    const R B0 = from_d<R>(p.B[0]), B1 = from_d<R>(p.B[1]), B2 = from_d<R>(p.B[2]);
    R a1[3], a2[3], a3[3], a4[3], u2[3], u3[3], u4[3];
    const R hh = R(0.5) * hs;
    a1[0] = kq * mfma(u[1], B2, -(u[2] * B1));
    a1[1] = kq * mfma(u[2], B0, -(u[0] * B2));
    a1[2] = kq * mfma(u[0], B1, -(u[1] * B0));
#pragma unroll
    for (int i = 0; i < 3; ++i) u2[i] = mfma(hh, a1[i], u[i]);
    a2[0] = kq * mfma(u2[1], B2, -(u2[2] * B1));
    a2[1] = kq * mfma(u2[2], B0, -(u2[0] * B2));
    a2[2] = kq * mfma(u2[0], B1, -(u2[1] * B0));
#pragma unroll
    for (int i = 0; i < 3; ++i) u3[i] = mfma(hh, a2[i], u[i]);
    a3[0] = kq * mfma(u3[1], B2, -(u3[2] * B1));
    a3[1] = kq * mfma(u3[2], B0, -(u3[0] * B2));
    a3[2] = kq * mfma(u3[0], B1, -(u3[1] * B0));
#pragma unroll
    for (int i = 0; i < 3; ++i) u4[i] = mfma(hs, a3[i], u[i]);
    a4[0] = kq * mfma(u4[1], B2, -(u4[2] * B1));
    a4[1] = kq * mfma(u4[2], B0, -(u4[0] * B2));
    a4[2] = kq * mfma(u4[0], B1, -(u4[1] * B0));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R su = mfma(R(2), u3[i], mfma(R(2), u2[i], u[i])) + u4[i];
        const R sa = mfma(R(2), a3[i], mfma(R(2), a2[i], a1[i])) + a4[i];
        if constexpr (sizeof(R) == 8)
            xo[i] = fma(h6, su, x[i]);
        else
            xo[i] = x[i] + to_d(h6 * su);
        uo[i] = mfma(h6, sa, u[i]);
    }
    const auto nd = mdivisor(msqrt(mfma(uo[0], uo[0], mfma(uo[1], uo[1], uo[2] * uo[2]))));
#pragma unroll
    for (int i = 0; i < 3; ++i) uo[i] = mdiv(uo[i], nd);
}

// True when the chord from x (inside volume vol) to x1 cannot leave vol:
// x1 lies inside the volume by more than kChordMargin, and in the world
// vacuum the chord's bounding box also stays kChordMargin away from the
// layer stack.  nav_exit would then return t > 1 for this chord (the exact
// exit parameter exceeds 1 by at least margin/|c|, far above rounding), and
// for a straight step to x1 = x + s u (unit u) an exit distance above s by
// at least the margin, so skipping it changes no result.
constexpr double kChordMargin = 1e-6;  // cm

// A step in a field is n equal RK4 substeps: n = ceil(s / h_max) of s / n
// for a step limit s up to kMaxSubsteps h_max (and up to max_field_step);
// a longer step is exactly kMaxSubsteps substeps of h_max (the count is
// set, not recomputed from a rounded quotient) and ends without an
// interaction: it bounds the work of one step of a looping track.
constexpr int kMaxSubsteps = 100;

// Cylinders: both ends within the shell's end planes and inside the circle
// of radius r_out - margin (the disc is convex, so the whole chord is), and
// for a hollow shell every point of the chord outside r_in + margin (both
// ends, and the chord's closest approach to the axis when it lies between
// them).  The exit parameter of the quadratic is then > 1 by at least
// margin/|c|, while its rounding error is below 1e-9/|c| for radii up to
// several metres (the discriminant is at least a * 2 r margin).
template <int G, typename R>
__device__ __forceinline__ bool chord_inside(const Params<R>& p, int vol, const double x[3], const double x1[3])
{
    const double m = kChordMargin;
    if constexpr (G == kGeomCylinders) {
        if (!(x1[2] > -p.half_z + m && x1[2] < p.half_z - m)) return false;
        const double ro = p.zb[vol + 1] - m;
        const double q1 = x1[0] * x1[0] + x1[1] * x1[1];
        if (!(q1 < ro * ro)) return false;
        if (vol > 0) {
            const double ri = p.zb[vol] + m;
            const double ri2 = ri * ri;
            const double q0 = x[0] * x[0] + x[1] * x[1];
            if (!(q1 > ri2) || !(q0 > ri2)) return false;
            const double cx = x1[0] - x[0], cy = x1[1] - x[1];
            const double a = cx * cx + cy * cy, b = x[0] * cx + x[1] * cy;
            if (b < 0.0 && -b < a && !(q0 - b * mdiv(b, a) > ri2)) return false;
        }
        return true;
    }
    if (vol >= 0) {
        return x1[2] > p.zb[vol] + m && x1[2] < p.zb[vol + 1] - m && x1[0] > -p.hx + m && x1[0] < p.hx - m &&
               x1[1] > -p.hy + m && x1[1] < p.hy - m;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!(x1[a] > p.wlo[a] + m && x1[a] < p.whi[a] - m)) return false;
    const double lo[3] = {-p.hx - m, -p.hy - m, p.zb[0] - m};
    const double hi[3] = {p.hx + m, p.hy + m, p.zb[p.n_layers] + m};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double smin = x[a] < x1[a] ? x[a] : x1[a];
        const double smax = x[a] < x1[a] ? x1[a] : x[a];
        if (smax < lo[a] || smin > hi[a]) return true;  // separated along axis a
    }
    return false;
}

// The chord test of a layer (vol >= 0, layered geometry) as integer
// comparisons through ord_key, whose order is the numeric order of non-NaN
// values: the lateral bounds' keys are formed when the geometry is loaded
// (Params::kxy), the layer's two z bounds per substep (held across the
// substep loop they cost registers, and spills, in the mixed-precision
// kernel), each with the same sum chord_inside forms.  A NaN coordinate fails one of the two tests
// of its axis in both forms, so every decision equals chord_inside's.
struct LayerBox {
    long long zlo, zhi;
};

template <typename R>
__device__ __forceinline__ LayerBox layer_box(const Params<R>& p, int vol)
{
    return LayerBox{ord_key(p.zb[vol] + kChordMargin), ord_key(p.zb[vol + 1] - kChordMargin)};
}

template <typename R>
__device__ __forceinline__ bool inside_box(const Params<R>& p, const LayerBox& b, const double x1[3])
{
    const long long k0 = ord_key(x1[0]), k1 = ord_key(x1[1]), k2 = ord_key(x1[2]);
    return k2 > b.zlo && k2 < b.zhi && k0 > p.kxy[0] && k0 < p.kxy[1] && k1 > p.kxy[2] && k1 < p.kxy[3];
}

// n substeps of length hs (the caller derives both from h_max); the chord
// of each substep is tested against the current volume and a crossing at
// fraction f repeats the substep with h f, snapped onto the plane.
// Returns the path length; *evals counts the integrator evaluations.
template <int G, typename R>
__device__ __forceinline__ double propagate_field(const Params<R>& p, int charge, double pm, int vol, double x[3],
                                                  R u[3], int n, double hs, Exit* bnd, bool* crossed, int* evals)
{
    double kq = mdiv(charge * kFieldC, pm);
    double s = 0.0;
    *crossed = false;
    const R hsr = R(hs);
    const R h6 = mdiv(hsr, R(6));
    const bool boxed = G == kGeomLayers && vol >= 0;
    for (int i = 0; i < n; ++i) {
        double x1[3], c[3];
        R u1[3];
        rk4(p, R(kq), x, u, hsr, h6, x1, u1);
        *evals += 1;
        if (!(boxed ? inside_box(p, layer_box(p, vol), x1) : chord_inside<G>(p, vol, x, x1))) {
#pragma unroll
            for (int a = 0; a < 3; ++a) c[a] = x1[a] - x[a];
            Exit e = nav_exit<G>(p, vol, x, c);
            if (e.t <= 1.0) {
                double h2 = hs * e.t;
                const R h2r = R(h2);
                rk4(p, R(kq), x, u, h2r, mdiv(h2r, R(6)), x1, u1);
                *evals += 1;
                if (e.axis >= 0) x1[e.axis] = e.plane;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    x[a] = x1[a];
                    u[a] = u1[a];
                }
                s += h2;
                *bnd = e;
                *crossed = true;
                return s;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = x1[a];
            u[a] = u1[a];
        }
        s += hs;
    }
    return s;
}

// ------------------------------------------------------------------ kinematics
// rotate (sin t cos phi, sin t sin phi, cos t), given in the frame whose z
// axis is u, into the global frame
template <typename R>
__device__ __forceinline__ void rotate(const R u[3], R cost, R phi, R out[3])
{
    R sint = msqrt(mfmax(R(0), (R(1) - cost) * (R(1) + cost)));
    R a = sint * mcos(phi);
    R b = sint * msin(phi);
    R perp2 = u[0] * u[0] + u[1] * u[1];
    if (perp2 > R(1e-20)) {
        R up = msqrt(perp2);
        out[0] = mdiv(u[0] * u[2] * a - u[1] * b, up) + u[0] * cost;
        out[1] = mdiv(u[1] * u[2] * a + u[0] * b, up) + u[1] * cost;
        out[2] = -up * a + u[2] * cost;
    } else if (u[2] >= R(0)) {
        out[0] = a;
        out[1] = b;
        out[2] = cost;
    } else {
        out[0] = -a;
        out[1] = b;
        out[2] = -cost;
    }
}

// out = normalize(pa da - pb db); false if the difference vanishes
template <typename R>
__device__ __forceinline__ bool momentum_balance(R pa, const R da[3], R pb, const R db[3], R out[3])
{
    R v0 = pa * da[0] - pb * db[0];
    R v1 = pa * da[1] - pb * db[1];
    R v2 = pa * da[2] - pb * db[2];
    R n = msqrt(v0 * v0 + v1 * v1 + v2 * v2);
    if (!(n > R(0))) return false;
    const auto nd = mdivisor(n);
    out[0] = mdiv(v0, nd);
    out[1] = mdiv(v1, nd);
    out[2] = mdiv(v2, nd);
    return true;
}

// ------------------------------------------------------------------ samplers
// Products of one interaction: up to two secondaries; `local` is energy
// deposited on the spot (binding energy).
template <typename R>
struct Products {
    int n;
    int type[2];
    R T[2];
    R dir[2][3];
    R local;
    bool parent_alive;
};

// Compton (Klein-Nishina): composition of the 1/eps and eps densities on
// [eps0, 1], eps0 = 1/(1 + 2 kappa), weights ln(1/eps0) and (1 - eps0^2)/2,
// rejection g = 1 - eps sin^2 / (1 + eps^2) (Butcher & Messel 1960).
template <typename R>
__device__ __forceinline__ void sample_compton(Draws& d, R k, R dir[3], Products<R>& out, R& knew)
{
    const R me = R(kMe);
    R kappa = mdiv(k, me);
    R eps0 = mdiv(R(1), R(1) + R(2) * kappa);
    R eps0sq = eps0 * eps0;
    R a1 = -mlog(eps0);
    R a2 = R(0.5) * (R(1) - eps0sq);
    R eps, epssq, onecost, sint2, g;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d), u3 = draw<R>(d);
        if (mdiv(a1, a1 + a2) > u1) {
            eps = mexp(-a1 * u2);
            epssq = eps * eps;
        } else {
            epssq = eps0sq + (R(1) - eps0sq) * u2;
            eps = msqrt(epssq);
        }
        onecost = mdiv(R(1) - eps, eps * kappa);
        sint2 = onecost * (R(2) - onecost);
        g = R(1) - mdiv(eps * sint2, R(1) + epssq);
        if (u3 <= g || trial >= kMaxTrials) break;
    }
    R phi = R(2.0 * kPi) * draw<R>(d);
    R cost = R(1) - onecost;
    R kp = eps * k;
    R gdir[3];
    rotate(dir, cost, phi, gdir);
    out.n = 0;
    R Te = k - kp;
    R edir[3];
    if (Te > R(0) && momentum_balance(k, dir, kp, gdir, edir)) {
        out.type[0] = 1;
        out.T[0] = Te;
        out.dir[0][0] = edir[0];
        out.dir[0][1] = edir[1];
        out.dir[0][2] = edir[2];
        out.n = 1;
    } else {
        out.local += Te;
    }
    dir[0] = gdir[0];
    dir[1] = gdir[1];
    dir[2] = gdir[2];
    knew = kp;
    out.parent_alive = true;
}

// Bethe-Heitler, complete screening: x = E(e-)/k uniform on
// [me/k, 1 - me/k], accepted with 1 - 4/3 x (1 - x); leptons collinear
// Dipole angular distribution of a particle emitted by a lepton of kinetic
// energy T (physics option kProcAngular): dN/dcos ~ (1 - beta cos)^-2,
// sampled by inverting its cumulative distribution,
// 1 - cos = 2 a (1 - u) / (a + 2 beta u) with a = 1 - beta = me^2/(E(E+p)).
template <typename R>
__device__ __forceinline__ R dipole_one_minus_cos(R T, R u)
{
    const R me = R(kMe);
    R E = T + me;
    R p = msqrt(T * (T + R(2) * me));
    R beta = mdiv(p, E);
    R a = mdiv(me * me, E * (E + p));
    return mdiv(R(2) * a * (R(1) - u), a + R(2) * beta * u);
}

template <typename R>
__device__ __forceinline__ void emit_dir(const R dir[3], R omc, R phi, R out[3])
{
    R cost = R(1) - omc;
    if (cost < R(-1)) cost = R(-1);
    rotate(dir, cost, phi, out);
}

// Rayleigh scattering (physics option kProcRayleigh): Thomson scattering
// off the atom with the form factor of an exponentially screened charge,
// F = Z / (1 + (q a)^2)^2, a = 0.88534 a0 Z^(-1/3).  With x = 1 - cos and
// b = 2 (k a / hbar c)^2 the angle density is (1 + (1 - x)^2) / (1 + b x)^4
// on [0, 2]: x from (1 + b x)^-4 by inversion, (1 + b x)^-3 = 1 - u (1 -
// (1 + 2b)^-3) (log1p/expm1 forms, exact for small b), accepted with
// (1 + (1 - x)^2) / 2.  The photon keeps its energy.
template <typename R>
__device__ __forceinline__ void sample_rayleigh(Draws& d, R k, R a_screen, R dir[3])
{
    R y = mdiv(k * a_screen, R(kHbarC));
    R b = R(2) * y * y;
    R tail = -mexpm1(R(-3) * mlog1p(R(2) * b));
    R x;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        x = mdiv(mexpm1(mdiv(-mlog1p(-u1 * tail), R(3))), b);
        if (x > R(2)) x = R(2);
        if (R(2) * u2 <= R(2) - R(2) * x + x * x || trial >= kMaxTrials) break;
    }
    R phi = R(2.0 * kPi) * draw<R>(d);
    R out[3];
    R cost = R(1) - x;
    rotate(dir, cost, phi, out);
#pragma unroll
    for (int a = 0; a < 3; ++a) dir[a] = out[a];
}

// Photoelectron angle (physics option kProcAngular): Sauter's K-shell
// distribution, dN/dcos ~ sin^2 / (1 - beta cos)^4 [1 + g (1 - beta cos)],
// g = gamma (gamma - 1) (gamma - 2) / 2.  In v = 1 - beta cos on [a, 2 - a]
// (a = 1 - beta) the density f(v) = (v - a)(2 - a - v)(1 + g v) / v^4 is
// bounded by 16 [(v + a)^-3 + max(g, 0) (v + a)^-2], whose two terms invert
// in closed form.  Returns 1 - cos = (v - a) / beta; isotropic below beta =
// 1e-3.
template <typename R>
__device__ __forceinline__ R sauter_one_minus_cos(Draws& d, R T)
{
    const R me = R(kMe);
    R E = T + me;
    R p = msqrt(T * (T + R(2) * me));
    R beta = mdiv(p, E);
    if (!(beta > R(1e-3))) return R(2) * draw<R>(d);
    R gam = mdiv(E, me);
    R a = mdiv(me * me, E * (E + p));
    R g = R(0.5) * gam * (gam - R(1)) * (gam - R(2));
    R gp = g > R(0) ? g : R(0);
    R i2a = mdiv(R(1), R(2) * a);
    R w1 = R(0.5) * (i2a * i2a - R(0.25)), w2 = gp * (i2a - R(0.5));
    R v = a;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d), u3 = draw<R>(d);
        if (u1 * (w1 + w2) < w1) {
            R w = i2a * i2a * (R(1) - u2) + R(0.25) * u2;
            v = mdiv(R(1), msqrt(w)) - a;
        } else {
            R w = i2a * (R(1) - u2) + R(0.5) * u2;
            v = mdiv(R(1), w) - a;
        }
        R va = v + a;
        R f = mdiv((v - a) * (R(2) - a - v) * (R(1) + g * v), v * v * v * v);
        R env = R(16) * (mdiv(R(1), va * va * va) + mdiv(gp, va * va));
        if (u3 * env <= f || trial >= kMaxTrials) break;
    }
    return mdiv(v - a, beta);
}

// Highland's width of the projected multiple-scattering angle (PDG review
// "Passage of particles through matter", Eq. 34.15, unit charge) after a
// path s at kinetic energy T; 0 where its bracket turns negative
template <typename R>
__device__ __forceinline__ R highland(R T, R s, R x0)
{
    R p = msqrt(T * (T + R(2) * R(kMe)));
    R beta = mdiv(p, T + R(kMe));
    R t = mdiv(s, x0);
    R f = R(1) + R(0.038) * mlog(mdiv(t, beta * beta));
    if (!(f > R(0))) return R(0);
    return mdiv(R(13.6), beta * p) * msqrt(t) * f;
}

// multiple scattering at the end of a step: space angle theta0 sqrt(-2 ln
// u_a) (two Gaussian projections of width theta0), capped at pi, azimuth
// 2 pi u_b, from draws kMscDraw and kMscDraw + 1 of the step.  Not inlined:
// the step kernel pays for it only when the option is on.
template <typename R>
__device__ __noinline__ void msc_deflect(Draws& d, R T, R s, R x0, R u[3])
{
    const R th0 = highland(T, s, x0);
    if (!(th0 > R(0))) return;
    d.next = kMscDraw;
    R ua = draw<R>(d), ub = draw<R>(d);
    R th = th0 * msqrt(R(-2) * mlog(ua));
    if (th > R(kPi)) th = R(kPi);
    R out[3];
    rotate(u, mcos(th), R(2.0 * kPi) * ub, out);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = out[a];
}

template <typename R>
__device__ __forceinline__ void sample_pair(Draws& d, R k, const R dir[3], Products<R>& out, bool angular)
{
    const R me = R(kMe);
    R eps0 = mdiv(me, k);
    R w = R(1) - R(2) * eps0;
    R x;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        x = eps0 + w * u1;
        R f = R(1) - R(4.0 / 3.0) * x * (R(1) - x);
        if (u2 <= f || trial >= kMaxTrials) break;
    }
    R Tm = x * k - me;
    if (Tm < R(0)) Tm = R(0);
    R Tp = (k - Tm) - R(2) * me;
    if (Tp < R(0)) Tp = R(0);
    out.n = 2;
    out.type[0] = 1;
    out.T[0] = Tm;
    out.type[1] = 2;
    out.T[1] = Tp;
    if (angular) {
        // each lepton at its own dipole angle, azimuths phi and phi + pi
        R um = draw<R>(d);
        R phi = R(2.0 * kPi) * draw<R>(d);
        R up = draw<R>(d);
        emit_dir(dir, dipole_one_minus_cos(Tm, um), phi, out.dir[0]);
        emit_dir(dir, dipole_one_minus_cos(Tp, up), phi + R(kPi), out.dir[1]);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out.dir[0][a] = dir[a];
            out.dir[1][a] = dir[a];
        }
    }
    out.parent_alive = false;
}

// photoelectric stand-in: photoelectron T = k - bk along the photon
template <typename R>
__device__ __forceinline__ void sample_photo(Draws& d, R k, R bk, const R dir[3], Products<R>& out, bool angular)
{
    out.n = 1;
    out.type[0] = 1;
    out.T[0] = k - bk;
    if (angular) {
        R omc = sauter_one_minus_cos(d, k - bk);
        R phi = R(2.0 * kPi) * draw<R>(d);
        emit_dir(dir, omc, phi, out.dir[0]);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) out.dir[0][a] = dir[a];
    }
    out.local += bk;
    out.parent_alive = false;
}

// bremsstrahlung (Tsai complete screening): k = kc (T/kc)^u, accepted with
// (4/3 - 4/3 y + y^2) / (4/3), y = k/E; photon along the lepton
template <typename R>
__device__ __forceinline__ void sample_brems(Draws& d, R T, R kc, const R dir[3], Products<R>& out, R& Tnew,
                                             bool angular)
{
    R E = T + R(kMe);
    R lr = mlog(mdiv(T, kc));
    R k;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        k = kc * mexp(u1 * lr);
        R y = mdiv(k, E);
        R f = R(4.0 / 3.0) - R(4.0 / 3.0) * y + y * y;
        if (u2 * R(4.0 / 3.0) <= f || trial >= kMaxTrials) break;
    }
    out.n = 1;
    out.type[0] = 0;
    out.T[0] = k;
    if (angular) {
        // photon at the radiating lepton's dipole angle; the lepton keeps
        // its direction (the nucleus takes the recoil)
        R u = draw<R>(d);
        R phi = R(2.0 * kPi) * draw<R>(d);
        emit_dir(dir, dipole_one_minus_cos(T, u), phi, out.dir[0]);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) out.dir[0][a] = dir[a];
    }
    Tnew = T - k;
    out.parent_alive = true;
}

// delta ray at cos = sqrt(Td (T + 2me) / (T (Td + 2me))); parent by
// momentum balance
template <typename R>
__device__ __forceinline__ void delta_kinematics(Draws& d, R T, R Td, R dir[3], Products<R>& out, R& Tnew)
{
    const R me = R(kMe);
    R cost = msqrt(mdiv(Td * (T + R(2) * me), T * (Td + R(2) * me)));
    if (cost > R(1)) cost = R(1);
    R phi = R(2.0 * kPi) * draw<R>(d);
    R ddir[3];
    rotate(dir, cost, phi, ddir);
    R p0 = msqrt(T * (T + R(2) * me));
    R pd = msqrt(Td * (Td + R(2) * me));
    R ndir[3];
    if (momentum_balance(p0, dir, pd, ddir, ndir)) {
        dir[0] = ndir[0];
        dir[1] = ndir[1];
        dir[2] = ndir[2];
    }
    out.n = 1;
    out.type[0] = 1;
    out.T[0] = Td;
    out.dir[0][0] = ddir[0];
    out.dir[0][1] = ddir[1];
    out.dir[0][2] = ddir[2];
    Tnew = T - Td;
    out.parent_alive = true;
}

// Moller: eps = xc / (1 - u (1 - 2 xc)) (1/eps^2 envelope on [xc, 1/2]),
// accepted with eps^2 B(eps) / (2 + g1^2/4)
template <typename R>
__device__ __forceinline__ void sample_moller(Draws& d, R T, R cut, R dir[3], Products<R>& out, R& Tnew)
{
    const R me = R(kMe);
    R xc = mdiv(cut, T);
    R g = mdiv(T + me, me);
    R g1 = mdiv(g - R(1), g);
    R c = mdiv(R(2) * g - R(1), g * g);
    R gmax = R(2) + R(0.25) * g1 * g1;
    R eps;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        eps = mdiv(xc, R(1) - u1 * (R(1) - R(2) * xc));
        R q = mdiv(eps, R(1) - eps);
        R f = R(1) + q * q + g1 * g1 * eps * eps - c * q;
        if (u2 * gmax <= f || trial >= kMaxTrials) break;
    }
    delta_kinematics(d, T, eps * T, dir, out, Tnew);
}

// Bhabha: eps = xc / (1 - u (1 - xc)) (1/eps^2 envelope on [xc, 1]),
// accepted with beta^2 eps^2 times the bracket of dsigma/deps (<= 1)
template <typename R>
__device__ __forceinline__ void sample_bhabha(Draws& d, R T, R cut, R dir[3], Products<R>& out, R& Tnew)
{
    const R me = R(kMe);
    R xc = mdiv(cut, T);
    R g = mdiv(T + me, me);
    R y = mdiv(R(1), g + R(1));
    R y2 = y * y;
    R t = R(1) - R(2) * y;
    R b2 = mdiv(T * (T + R(2) * me), (T + me) * (T + me));
    R c1 = R(2) - y2;
    R c2 = t * (R(3) + y2);
    R c4 = t * t * t;
    R c3 = t * t + c4;
    R eps;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        eps = mdiv(xc, R(1) - u1 * (R(1) - xc));
        R f = R(1) - b2 * eps * (c1 - eps * (c2 - eps * (c3 - eps * c4)));
        if (u2 <= f || trial >= kMaxTrials) break;
    }
    delta_kinematics(d, T, eps * T, dir, out, Tnew);
}

// two-photon annihilation in flight (Heitler): eps = emin (emax/emin)^u
// (1/eps envelope), accepted with 1 - ((g+1)^2 eps + 1/eps)/(g^2 + 4g + 1);
// photon 1 at cos = (T + 2me)(E1 - me)/(p E1), photon 2 by momentum balance
template <typename R>
__device__ __forceinline__ void sample_annih(Draws& d, R T, const R dir[3], Products<R>& out)
{
    const R me = R(kMe);
    R tau = mdiv(T, me);
    R g = tau + R(1);
    R a = tau + R(2);
    R s = msqrt(tau * (tau + R(2)));
    R emin = R(0.5) * (R(1) - mdiv(s, a));
    R emax = R(1) - emin;
    R lr = mlog(mdiv(emax, emin));
    R bq = g * g + R(4) * g + R(1);
    R eps;
    for (int trial = 1;; ++trial) {
        R u1 = draw<R>(d), u2 = draw<R>(d);
        eps = emin * mexp(u1 * lr);
        R f = R(1) - mdiv(a * a * eps + mdiv(R(1), eps), bq);
        if (u2 <= f || trial >= kMaxTrials) break;
    }
    R Etot = T + R(2) * me;
    R E1 = eps * Etot;
    R E2 = Etot - E1;
    R pm = msqrt(T * (T + R(2) * me));
    R cost = mdiv(Etot * (E1 - me), pm * E1);
    if (cost > R(1)) cost = R(1);
    if (cost < R(-1)) cost = R(-1);
    R phi = R(2.0 * kPi) * draw<R>(d);
    R d1[3], d2[3];
    rotate(dir, cost, phi, d1);
    if (!momentum_balance(pm, dir, E1, d1, d2)) {
        d2[0] = -d1[0];
        d2[1] = -d1[1];
        d2[2] = -d1[2];
    }
    out.n = 2;
    out.type[0] = 0;
    out.T[0] = E1;
    out.type[1] = 0;
    out.T[1] = E2;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out.dir[0][a] = d1[a];
        out.dir[1][a] = d2[a];
    }
    out.parent_alive = false;
}

}  // namespace emt
