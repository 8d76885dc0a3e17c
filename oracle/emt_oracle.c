/*
 * emt_oracle.c -- plain, slow, FP64 CPU oracle of the per-step EM transport
 * loop described in arXiv:2203.09467 (Sec. 2.1 "one thread per track";
 * Sec. 2.2 physics, Table 1; Sec. 2.3 geometry and fields; Sec. 3.2
 * preliminary results).
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  Nothing in the GPU library calls,
 * links or includes it, and it includes nothing from the GPU library.
 *
 * The paper names models but prints no formula, so each function below
 * states the textbook closed form it writes out and where it comes from.
 * Parity status per function:
 *   pinned  : checked by tests against limits, identities, published
 *             constants, quadrature or brute force (see tests/).
 *   absolute agreement with measured data or Geant4 is "parity unpinned"
 *   (nothing in this repository can check it).
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add: the GPU FP64
 * path follows the same operation order and also disables contraction).
 */
#include "emt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ */
/* Constants: CODATA 2018                                              */
/* ------------------------------------------------------------------ */
#define ME 0.51099895             /* electron mass, MeV */
#define RE 2.8179403262e-13       /* classical electron radius, cm */
#define ALPHA (1.0 / 137.035999084)
#define NAVO 6.02214076e23        /* Avogadro, 1/mol */
#define PI 3.14159265358979323846
#define FIELD_C 2.99792458        /* q/p -> curvature: 1/(cm T) per 1/MeV */
#define BOHR 0.529177210903e-8    /* Bohr radius, cm (CODATA 2018) */
#define HBARC 197.3269804e-13     /* hbar c, MeV cm (CODATA 2018) */
#define INF_D (1.0 / 0.0)

/* ------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11.  Round: two 32x32->64 multiplies by     */
/* M0=0xD2511F53, M1=0xCD9E8D57; key schedule Weyl increments          */
/* W0=0x9E3779B9, W1=0xBB67AE85; 10 rounds.                            */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Stream keying (a reading; the paper's demo used XORWOW, Sec. 3.2 caveats):
 *   key = (lo32(event_id), hi32(event_id) ^ seed)
 *   ctr = (lo32(uid), hi32(uid), step, j >> 1)
 * draw j uses output words 2(j&1) (low) and 2(j&1)+1 (high) of that block;
 * the 64-bit word w gives u = ((w >> 12) + 1/2) * 2^-52, in (0,1).       */
static void track_key(uint32_t seed, uint64_t event_id, uint32_t key[2])
{
    key[0] = (uint32_t)event_id;
    key[1] = (uint32_t)(event_id >> 32) ^ seed;
}

double orc_track_uniform(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step, uint32_t j)
{
    uint32_t key[2], ctr[4], out[4];
    track_key(seed, event_id, key);
    ctr[0] = (uint32_t)uid;
    ctr[1] = (uint32_t)(uid >> 32);
    ctr[2] = step;
    ctr[3] = j >> 1;
    orc_philox4x32_10(ctr, key, out);
    uint64_t lo = out[2 * (j & 1u)], hi = out[2 * (j & 1u) + 1];
    uint64_t w = (hi << 32) | lo;
    return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

/* child k of (uid, step): key word 0 xor 0x5EC0DA7A, counter word 3 has the
 * top bit set so it never coincides with a draw block. */
uint64_t orc_child_uid(uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step, uint32_t k)
{
    uint32_t key[2], ctr[4], out[4];
    track_key(seed, event_id, key);
    key[0] ^= 0x5EC0DA7Au;
    ctr[0] = (uint32_t)uid;
    ctr[1] = (uint32_t)(uid >> 32);
    ctr[2] = step;
    ctr[3] = 0x80000000u + k;
    orc_philox4x32_10(ctr, key, out);
    return ((uint64_t)out[1] << 32) | (uint64_t)out[0];
}

typedef struct {
    uint32_t seed;
    uint64_t event_id;
    uint64_t uid;
    uint32_t step;
    uint32_t next; /* next draw index */
} draws_t;

static double draw(draws_t* d)
{
    double u = orc_track_uniform(d->seed, d->event_id, d->uid, d->step, d->next);
    d->next += 1;
    return u;
}

/* ------------------------------------------------------------------ */
/* Closed forms (all pinned by tests unless stated)                    */
/* ------------------------------------------------------------------ */

/* Radiation length, Tsai (Rev. Mod. Phys. 46 (1974) 815) as quoted in the
 * PDG review "Passage of particles through matter", Eq. 34.26:
 * 1/X0 = 4 alpha re^2 (NA/A) { Z^2 [Lrad - f(Z)] + Z L'rad },
 * Lrad = ln(184.15 Z^-1/3), L'rad = ln(1194 Z^-2/3) (Z >= 5),
 * f(Z) = a^2 [ 1/(1+a^2) + 0.20206 - 0.0369 a^2 + 0.0083 a^4 - 0.002 a^6 ],
 * a = alpha Z.  Returns X0 in g/cm^2. */
double orc_x0_gcm2(double Z, double A)
{
    double a = ALPHA * Z;
    double a2 = a * a;
    double fz = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
    double z13 = cbrt(Z);
    double lrad = log(184.15 / z13);
    double lprad = log(1194.0 / (z13 * z13));
    double inv = 4.0 * ALPHA * RE * RE * (NAVO / A) * (Z * Z * (lrad - fz) + Z * lprad);
    return 1.0 / inv;
}

/* Klein-Nishina total cross section per electron (Klein & Nishina 1929;
 * e.g. Heitler, "Quantum theory of radiation", Sec. 22), kappa = k/me:
 * sigma = 2 pi re^2 { (1+kappa)/kappa^2 [ 2(1+kappa)/(1+2kappa)
 *         - ln(1+2kappa)/kappa ] + ln(1+2kappa)/(2kappa)
 *         - (1+3kappa)/(1+2kappa)^2 }                                   */
double orc_sigma_kn(double k)
{
    double kappa = k / ME;
    double a = 1.0 + 2.0 * kappa;
    double l = log(a);
    double t1 = (1.0 + kappa) / (kappa * kappa) * (2.0 * (1.0 + kappa) / a - l / kappa);
    double t2 = l / (2.0 * kappa);
    double t3 = (1.0 + 3.0 * kappa) / (a * a);
    return 2.0 * PI * RE * RE * (t1 + t2 - t3);
}

/* KN differential in eps = k'/k: dsigma/deps = pi re^2 / kappa
 * (1/eps + eps) (1 - eps sin^2(theta)/(1+eps^2)), 1-cos = (1-eps)/(kappa eps) */
double orc_dsigma_kn_deps(double k, double eps)
{
    double kappa = k / ME;
    double onecost = (1.0 - eps) / (eps * kappa);
    double sint2 = onecost * (2.0 - onecost);
    return PI * RE * RE / kappa * (1.0 / eps + eps) * (1.0 - eps * sint2 / (1.0 + eps * eps));
}

/* Bethe-Heitler pair production with complete screening (PDG Eq. 34.31):
 * dsigma/dx = A/(X0 NA) [1 - 4/3 x(1-x)], x = E(e-)/k, restricted to the
 * kinematic range x in [me/k, 1 - me/k] (a reading).  With h = 1/2 - me/k,
 * the integral is 4h/3 + 8h^3/9 (-> 7/9 for k -> inf).                  */
double orc_sigma_pair_atom(double Z, double A, double k)
{
    if (k <= 2.0 * ME) return 0.0;
    double h = 0.5 - ME / k;
    double integral = 4.0 / 3.0 * h + 8.0 / 9.0 * h * h * h;
    return A / (orc_x0_gcm2(Z, A) * NAVO) * integral;
}

double orc_dsigma_pair_dx(double Z, double A, double k, double x)
{
    double eps0 = ME / k;
    if (x < eps0 || x > 1.0 - eps0) return 0.0;
    return A / (orc_x0_gcm2(Z, A) * NAVO) * (1.0 - 4.0 / 3.0 * x * (1.0 - x));
}

/* Photoelectric stand-in (Livermore data is not available): Sauter's
 * high-energy K-shell limit sigma_K = 4 pi re^2 alpha^4 Z^5 (me/k)
 * (Heitler Sec. 21; Davisson & Evans), times 5/4 for the outer shells;
 * zero at or below the K binding energy bk.                             */
double orc_sigma_photo_atom(double Z, double k, double bk)
{
    if (k <= bk) return 0.0;
    double a2 = ALPHA * ALPHA;
    double z5 = Z * Z * Z * Z * Z;
    return 5.0 * PI * RE * RE * (a2 * a2) * z5 * (ME / k);
}

/* Moller cross section per electron, eps = T_delta/T in [xc, 1/2]
 * (Moller 1932; form as in ICRU 37 and the Geant4 physics reference):
 * dsigma/deps = 2 pi re^2 me / (beta^2 T) [ 1/eps^2 + 1/(1-eps)^2
 *     + ((g-1)/g)^2 - (2g-1)/g^2 / (eps (1-eps)) ]                       */
double orc_dsigma_moller_deps(double T, double eps)
{
    double g = (T + ME) / ME;
    double b2 = T * (T + 2.0 * ME) / ((T + ME) * (T + ME));
    double g1 = (g - 1.0) / g;
    double c = (2.0 * g - 1.0) / (g * g);
    double br = 1.0 / (eps * eps) + 1.0 / ((1.0 - eps) * (1.0 - eps)) + g1 * g1 - c / (eps * (1.0 - eps));
    return 2.0 * PI * RE * RE * ME / (b2 * T) * br;
}

/* integral of the above over [xc, 1/2], xc = cut/T (needs T > 2 cut):
 * g1^2 (1/2 - xc) + 1/xc - 1/(1-xc) - c ln((1-xc)/xc)                  */
double orc_sigma_moller(double T, double cut)
{
    if (T <= 2.0 * cut) return 0.0;
    double xc = cut / T;
    double g = (T + ME) / ME;
    double b2 = T * (T + 2.0 * ME) / ((T + ME) * (T + ME));
    double g1 = (g - 1.0) / g;
    double c = (2.0 * g - 1.0) / (g * g);
    double br = g1 * g1 * (0.5 - xc) + 1.0 / xc - 1.0 / (1.0 - xc) - c * log((1.0 - xc) / xc);
    return 2.0 * PI * RE * RE * ME / (b2 * T) * br;
}

/* Bhabha cross section per electron (Bhabha 1936; ICRU 37 form),
 * eps = T_delta/T in [xc, 1], y = 1/(g+1):
 * dsigma/deps = 2 pi re^2 me / T [ 1/(beta^2 eps^2) - B1/eps + B2
 *               - B3 eps + B4 eps^2 ],
 * B1 = 2 - y^2, B2 = (1-2y)(3+y^2), B4 = (1-2y)^3, B3 = (1-2y)^2 + B4.  */
static void bhabha_coeffs(double T, double* b2, double* c1, double* c2, double* c3, double* c4)
{
    double g = (T + ME) / ME;
    double y = 1.0 / (g + 1.0);
    double y2 = y * y;
    double t = 1.0 - 2.0 * y;
    *b2 = T * (T + 2.0 * ME) / ((T + ME) * (T + ME));
    *c1 = 2.0 - y2;
    *c2 = t * (3.0 + y2);
    *c4 = t * t * t;
    *c3 = t * t + *c4;
}

double orc_dsigma_bhabha_deps(double T, double eps)
{
    double b2, c1, c2, c3, c4;
    bhabha_coeffs(T, &b2, &c1, &c2, &c3, &c4);
    double br = 1.0 / (b2 * eps * eps) - c1 / eps + c2 - c3 * eps + c4 * eps * eps;
    return 2.0 * PI * RE * RE * ME / T * br;
}

double orc_sigma_bhabha(double T, double cut)
{
    if (T <= cut) return 0.0;
    double xc = cut / T;
    double b2, c1, c2, c3, c4;
    bhabha_coeffs(T, &b2, &c1, &c2, &c3, &c4);
    double br = (1.0 / xc - 1.0) / b2 + c1 * log(xc) + c2 * (1.0 - xc) - c3 * (1.0 - xc * xc) / 2.0 +
                c4 * (1.0 - xc * xc * xc) / 3.0;
    return 2.0 * PI * RE * RE * ME / T * br;
}

/* Two-photon annihilation in flight, Heitler (Quantum theory of radiation,
 * Sec. 29), per target electron, tau = T/me, g = tau + 1:
 * sigma = pi re^2/(g+1) [ (g^2+4g+1)/(g^2-1) ln(g + sqrt(g^2-1))
 *         - (g+3)/sqrt(g^2-1) ]                                          */
double orc_sigma_heitler(double T)
{
    double tau = T / ME;
    double g = tau + 1.0;
    double gg1 = tau * (tau + 2.0); /* g^2 - 1 */
    double s = sqrt(gg1);
    return PI * RE * RE / (g + 1.0) * ((g * g + 4.0 * g + 1.0) / gg1 * log(g + s) - (g + 3.0) / s);
}

/* Differential in the energy fraction eps of one photon, eps in
 * [emin, 1-emin], emin = (1 - sqrt((g-1)/(g+1)))/2:
 * dsigma/deps = pi re^2 / ((g+1)(g^2-1)) S(eps),
 * S(eps) = -(g+1)^2 + (g^2+4g+1)/eps - 1/eps^2.  Integrates to the total
 * above (checked by quadrature in the tests).                           */
double orc_dsigma_heitler_deps(double T, double eps)
{
    double tau = T / ME;
    double g = tau + 1.0;
    double a = g + 1.0;
    double gg1 = tau * (tau + 2.0);
    double s = sqrt(gg1);
    double emin = 0.5 * (1.0 - s / a);
    if (eps < emin || eps > 1.0 - emin) return 0.0;
    double S = -a * a + (g * g + 4.0 * g + 1.0) / eps - 1.0 / (eps * eps);
    return PI * RE * RE / (a * gg1) * S;
}

/* Bremsstrahlung, complete screening (Tsai 1974; PDG Eq. 34.29 without the
 * small y^2/9 term): dSigma/dk = 1/(X0 k) (4/3 - 4/3 y + y^2), y = k/E,
 * E = T + me, k <= T.  Discrete part k in (kc, T]:
 * Sigma = 1/X0 [ 4/3 ln(T/kc) - 4/3 (T-kc)/E + (T^2 - kc^2)/(2E^2) ].   */
/* Rayleigh (coherent) scattering, process bit ORC_RAYLEIGH (Table 1 uses
 * Livermore form factors, which are not available): Thomson scattering off
 * the atom with the form factor of an exponentially screened charge,
 * F(q) = Z / (1 + (q a)^2)^2, a = 0.88534 a0 Z^(-1/3) (the Thomas-Fermi
 * radius).  With x = 1 - cos(theta), (q a)^2 = b x, b = 2 (k a / hbar c)^2:
 * dsigma/dx = pi re^2 Z^2 (1 + (1 - x)^2) / (1 + b x)^4 on [0, 2].
 * The integral I(b) = int_0^2 (2 - 2x + x^2) (1 + b x)^-4 dx is summed as
 * its Taylor series below b = 0.1 (the closed form cancels there) and in
 * closed form above: with y = 1 + b x, Y = 1 + 2 b,
 * I = [A (1 - Y^-3)/3 + B (1 - Y^-2)/2 + C (1 - Y^-1)] / b,
 * A = 2 + 2/b + 1/b^2, B = -2/b - 2/b^2, C = 1/b^2. */
static double rayleigh_b(double Z, double k)
{
    double a = 0.88534 * BOHR / cbrt(Z);
    double y = k * a / HBARC;
    return 2.0 * y * y;
}

static double rayleigh_integral(double b)
{
    if (b < 0.1) {
        /* sum_n (-1)^n C(n+3,3) b^n m_n, m_n = int_0^2 (2 - 2x + x^2) x^n dx */
        double sum = 0.0, bn = 1.0, p2 = 4.0; /* p2 = 2^(n+2) */
        for (int n = 0; n < 40; ++n) {
            double mn = p2 / (n + 1.0) - 2.0 * p2 / (n + 2.0) + 2.0 * p2 / (n + 3.0);
            double c = (n + 1.0) * (n + 2.0) * (n + 3.0) / 6.0;
            sum += ((n & 1) ? -c : c) * bn * mn;
            bn *= b;
            p2 *= 2.0;
        }
        return sum;
    }
    double Y = 1.0 + 2.0 * b;
    double A = 2.0 + 2.0 / b + 1.0 / (b * b), B = -2.0 / b - 2.0 / (b * b), C = 1.0 / (b * b);
    double y1 = 1.0 / Y, y2 = y1 * y1, y3 = y2 * y1;
    return (A * (1.0 - y3) / 3.0 + B * (1.0 - y2) / 2.0 + C * (1.0 - y1)) / b;
}

double orc_sigma_rayleigh_atom(double Z, double k)
{
    return PI * RE * RE * Z * Z * rayleigh_integral(rayleigh_b(Z, k));
}

double orc_dsigma_rayleigh_dx(double Z, double k, double x)
{
    double b = rayleigh_b(Z, k);
    double d = 1.0 + b * x;
    return PI * RE * RE * Z * Z * (2.0 - 2.0 * x + x * x) / (d * d * d * d);
}

double orc_sigma_brems_macro(double x0_cm, double T, double kc)
{
    if (T <= kc) return 0.0;
    double E = T + ME;
    return 1.0 / x0_cm *
           (4.0 / 3.0 * log(T / kc) - 4.0 / 3.0 * (T - kc) / E + (T * T - kc * kc) / (2.0 * E * E));
}

double orc_dsigma_brems_macro_dk(double x0_cm, double T, double k)
{
    double E = T + ME;
    double y = k / E;
    return 1.0 / (x0_cm * k) * (4.0 / 3.0 - 4.0 / 3.0 * y + y * y);
}

/* radiative loss below the cut, k' = min(kc, T):
 * S_rad = 1/X0 [ 4/3 k' - 2/3 k'^2/E + k'^3/(3E^2) ]                     */
double orc_dedx_rad(double x0_cm, double T, double kc)
{
    double E = T + ME;
    double kp = kc < T ? kc : T;
    return 1.0 / x0_cm * (4.0 / 3.0 * kp - 2.0 / 3.0 * kp * kp / E + kp * kp * kp / (3.0 * E * E));
}

/* Restricted collision stopping power, Berger & Seltzer (NBSIR 82-2550;
 * ICRU 37, Eqs. 2.2-2.4 with the restriction of Geant4 PRM Sec. 10.1):
 * S = 2 pi re^2 me n_el / beta^2 [ ln(2(tau+2)/(I/me)^2) + F(tau,D) - delta ]
 * e-: D = min(cut, T/2)/me,
 *     F = -1 - b2 + ln((tau-D) D) + tau/(tau-D)
 *         + [D^2/2 + (2tau+1) ln(1 - D/tau)]/g^2
 * e+: D = min(cut, T)/me, y = 1/(tau+2),
 *     F = ln(tau D) - b2/tau [tau + 2D - 3/2 D^2 y - (D - D^3/3) y^2
 *         - (D^2/2 - tau D^3/3 + D^4/4) y^3]
 * density effect: high-energy asymptote (Sternheimer; PDG Eq. 34.6)
 * delta = max(0, 2 ln(beta g) + 2 ln(hw_p/I) - 1),
 * hw_p = 28.816 sqrt(rho Z/A) eV.  Floored at 1e-12 MeV/cm.              */
double orc_dedx_coll(double Z, double A, double rho, double I_eV, int charge, double T, double cut)
{
    double nel = rho * NAVO / A * Z;
    double tau = T / ME;
    double g = tau + 1.0;
    double b2 = tau * (tau + 2.0) / (g * g);
    double Im = I_eV * 1e-6 / ME;
    double F;
    if (charge < 0) {
        double dmax = 0.5 * T;
        double D = (cut < dmax ? cut : dmax) / ME;
        F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D) +
            (0.5 * D * D + (2.0 * tau + 1.0) * log(1.0 - D / tau)) / (g * g);
    } else {
        double D = (cut < T ? cut : T) / ME;
        double y = 1.0 / (tau + 2.0);
        double D2 = D * D, D3 = D2 * D, D4 = D3 * D;
        double y2 = y * y, y3 = y2 * y;
        F = log(tau * D) - b2 / tau *
                               (tau + 2.0 * D - 1.5 * D2 * y - (D - D3 / 3.0) * y2 -
                                (0.5 * D2 - tau * D3 / 3.0 + 0.25 * D4) * y3);
    }
    double hwp = 28.816 * sqrt(rho * Z / A); /* eV */
    double bg = sqrt(tau * (tau + 2.0));
    double delta = 2.0 * log(bg) + 2.0 * log(hwp / I_eV) - 1.0;
    if (delta < 0.0) delta = 0.0;
    double S = 2.0 * PI * RE * RE * ME * nel / b2 * (log(2.0 * (tau + 2.0) / (Im * Im)) + F - delta);
    if (S < 1e-12) S = 1e-12;
    return S;
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n
 * (Abramowitz & Stegun 25.4.29): P_n by the three-term recurrence,
 * P'_n = n (x P_n - P_{n-1})/(x^2-1), w = 2/((1-x^2) P'_n^2).            */
void orc_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged root */
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z; /* ascending */
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------ */
/* Handle: materials, tables, geometry                                 */
/* ------------------------------------------------------------------ */
#define MAXMAT 16
#define MAXLAYER 4096
#define NQ 5

typedef struct {
    double Z, A, rho, I_eV, bk;
    int vacuum;
    double n_at, n_el, x0_cm;
} mat_t;

struct orc_handle {
    int n_mat;
    mat_t mat[MAXMAT];
    double cut[3]; /* gamma, e-, e+ */
    double e_lo, e_hi;
    int bpd, n_grid;
    double step_frac, final_range;
    unsigned mask;
    double* grid;  /* n_grid */
    double* igrid; /* n_grid: 1 / (grid[i+1] - grid[i]) (last entry unused) */
    double* irs;   /* [mat][particle 3][n_grid]: 1 / (R[i+1] - R[i]) of the range tables */
    double* table; /* [mat][particle 3][q NQ][n_grid] */
    /* geometry */
    int n_layers;
    int layer_mat[MAXLAYER];
    int layer_bin[MAXLAYER];
    double zb[MAXLAYER + 1];
    double hx, hy;
    double wlo[3], whi[3];
    double B[3];
    double rk_delta;
    int max_steps;
    int n_bins;
    double max_field_step;
    int has_field;
    int geom;      /* GEOM_LAYERS or GEOM_CYLINDERS */
    double half_z; /* cylinders: the stack spans |z| <= half_z */
    int score_z;   /* 1: histogram bins along z; 0: bins per volume */
    double zs_lo, zs_scale; /* z bin = floor((z - zs_lo) * zs_scale) */
    uint32_t seed;
};

static double* tab(const orc_handle* h, int m, int p, int q)
{
    return h->table + (((size_t)m * 3 + p) * NQ + q) * h->n_grid;
}

/* restricted total stopping power used for the range tables */
static double dedx_total(const orc_handle* h, const mat_t* m, int p, double T)
{
    double cut_e = h->cut[1];
    double coll = orc_dedx_coll(m->Z, m->A, m->rho, m->I_eV, p == 1 ? -1 : 1, T, cut_e);
    return coll + orc_dedx_rad(m->x0_cm, T, h->cut[0]);
}

static void build_tables(orc_handle* h)
{
    int n = h->n_grid;
    for (int i = 0; i < n; ++i) h->grid[i] = h->e_lo * pow(10.0, (double)i / h->bpd);
    for (int i = 0; i + 1 < n; ++i) h->igrid[i] = 1.0 / (h->grid[i + 1] - h->grid[i]);
    double glx[16], glw[16];
    orc_gauss_legendre(16, glx, glw);
    for (int mi = 0; mi < h->n_mat; ++mi) {
        mat_t* m = &h->mat[mi];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < NQ; ++q) memset(tab(h, mi, p, q), 0, sizeof(double) * n);
        if (m->vacuum) continue;
        double kc = h->cut[0], cut_e = h->cut[1];
        for (int i = 0; i < n; ++i) {
            double E = h->grid[i];
            /* photons */
            if (h->mask & ORC_PHOTO) tab(h, mi, 0, 0)[i] = m->n_at * orc_sigma_photo_atom(m->Z, E, m->bk);
            if (h->mask & ORC_COMPTON) tab(h, mi, 0, 1)[i] = m->n_el * orc_sigma_kn(E);
            if (h->mask & ORC_PAIR) {
                double s = 0.0;
                if (E > 2.0 * ME) {
                    double hh = 0.5 - ME / E;
                    s = (4.0 / 3.0 * hh + 8.0 / 9.0 * hh * hh * hh) / m->x0_cm;
                }
                tab(h, mi, 0, 2)[i] = s;
            }
            if (h->mask & ORC_RAYLEIGH) tab(h, mi, 0, 3)[i] = m->n_at * orc_sigma_rayleigh_atom(m->Z, E);
            /* electrons */
            if (h->mask & ORC_IONI) tab(h, mi, 1, 0)[i] = m->n_el * orc_sigma_moller(E, cut_e);
            if (h->mask & ORC_BREMS) tab(h, mi, 1, 1)[i] = orc_sigma_brems_macro(m->x0_cm, E, kc);
            tab(h, mi, 1, 4)[i] = dedx_total(h, m, 1, E);
            /* positrons */
            if (h->mask & ORC_IONI) tab(h, mi, 2, 0)[i] = m->n_el * orc_sigma_bhabha(E, cut_e);
            if (h->mask & ORC_BREMS) tab(h, mi, 2, 1)[i] = orc_sigma_brems_macro(m->x0_cm, E, kc);
            if (h->mask & ORC_ANNIH) tab(h, mi, 2, 2)[i] = m->n_el * orc_sigma_heitler(E);
            tab(h, mi, 2, 4)[i] = dedx_total(h, m, 2, E);
        }
        /* range: R_0 = E_0/S(E_0); R_i = R_{i-1} + int dE/S over
         * [E_{i-1}, E_i], 16-point Gauss-Legendre in u = ln E with
         * integrand E/S(E) evaluated from the closed form (not the table).
         * Each interval is split at the energies where S has a kink, in
         * ascending order: the restriction switch (2 cut for e-, cut for
         * e+), the radiative cut kc, and the onset of the density effect,
         * beta*gamma = e^(1/2) I / hw_p. */
        double hwp = 28.816 * sqrt(m->rho * m->Z / m->A);
        double bg0 = exp(0.5) * m->I_eV / hwp;
        double t_dens = ME * (sqrt(1.0 + bg0 * bg0) - 1.0);
        for (int p = 1; p < 3; ++p) {
            double* R = tab(h, mi, p, 3);
            double kinks[3] = {p == 1 ? 2.0 * cut_e : cut_e, kc, t_dens};
            for (int x = 0; x < 3; ++x) /* sort ascending (3 elements) */
                for (int y = x + 1; y < 3; ++y)
                    if (kinks[y] < kinks[x]) {
                        double t = kinks[x];
                        kinks[x] = kinks[y];
                        kinks[y] = t;
                    }
            R[0] = h->grid[0] / tab(h, mi, p, 4)[0];
            for (int i = 1; i < n; ++i) {
                double edges[5];
                int ne = 0;
                edges[ne++] = h->grid[i - 1];
                for (int x = 0; x < 3; ++x)
                    if (kinks[x] > edges[ne - 1] && kinks[x] < h->grid[i]) edges[ne++] = kinks[x];
                edges[ne++] = h->grid[i];
                double acc = 0.0;
                for (int sub = 0; sub + 1 < ne; ++sub) {
                    double a = log(edges[sub]), b = log(edges[sub + 1]);
                    double half = 0.5 * (b - a), mid = 0.5 * (a + b);
                    double sum = 0.0;
                    for (int j = 0; j < 16; ++j) {
                        double E = exp(mid + half * glx[j]);
                        sum += glw[j] * (E / dedx_total(h, m, p, E));
                    }
                    acc += half * sum;
                }
                R[i] = R[i - 1] + acc;
            }
            double* irs = h->irs + ((size_t)mi * 3 + p) * n;
            for (int i = 0; i + 1 < n; ++i) irs[i] = 1.0 / (R[i + 1] - R[i]);
        }
    }
}

/* index n with grid[n] <= E < grid[n+1], clamped to [0, n_grid-2]
 * (plain scan: the definition, no logarithm) */
static int find_bin(const orc_handle* h, double E)
{
    int n = 0;
    while (n + 1 < h->n_grid - 1 && h->grid[n + 1] <= E) ++n;
    return n;
}

/* piecewise linear in E between nodes; constant outside the grid.  The
 * fraction within an interval is (E - E_n) times the interval's reciprocal
 * width, rounded once when the grid is built, and v_n + (v_{n+1} - v_n) f
 * is one fused multiply-add (a reading: the paper fixes no interpolation
 * arithmetic; a product instead of a quotient per lookup, one rounding
 * instead of two).  The straight-line move x + s u is fused likewise. */
static double lookup(const orc_handle* h, const double* v, double E)
{
    if (E <= h->grid[0]) return v[0];
    if (E >= h->grid[h->n_grid - 1]) return v[h->n_grid - 1];
    int n = find_bin(h, E);
    double f = (E - h->grid[n]) * h->igrid[n];
    return fma(v[n + 1] - v[n], f, v[n]);
}

/* range: linear through the origin below the first node, linear between
 * nodes, extrapolated with the last slope above the grid */
static double range_of(const orc_handle* h, const double* R, double T)
{
    if (T < h->grid[0]) return R[0] * (T / h->grid[0]);
    int n = find_bin(h, T);
    double f = (T - h->grid[n]) * h->igrid[n];
    return fma(R[n + 1] - R[n], f, R[n]);
}

/* inverse of range_of (the same piecewise-linear function, inverted with
 * the range intervals' reciprocal widths irs) */
static double inv_range_of(const orc_handle* h, const double* R, const double* irs, double r)
{
    if (r < R[0]) return h->grid[0] * (r / R[0]);
    int n = 0;
    while (n + 1 < h->n_grid - 1 && R[n + 1] <= r) ++n;
    double f = (r - R[n]) * irs[n];
    return fma(h->grid[n + 1] - h->grid[n], f, h->grid[n]);
}

static const double* irs_of(const orc_handle* h, int m, int p) { return h->irs + ((size_t)m * 3 + p) * h->n_grid; }

double orc_range(const orc_handle* h, int m, int ci, double T)
{
    return range_of(h, tab(h, m, ci, 3), T);
}

double orc_inv_range(const orc_handle* h, int m, int ci, double r)
{
    return inv_range_of(h, tab(h, m, ci, 3), irs_of(h, m, ci), r);
}

orc_handle* orc_create(const double* materials, int n_mat, const double* physics, const double* layers,
                       int n_layers, const double* world, uint32_t seed)
{
    if (n_mat < 0 || n_mat > MAXMAT || n_layers < 1 || n_layers > MAXLAYER) return NULL;
    orc_handle* h = (orc_handle*)calloc(1, sizeof(orc_handle));
    h->n_mat = n_mat;
    for (int i = 0; i < n_mat; ++i) {
        mat_t* m = &h->mat[i];
        m->Z = materials[5 * i + 0];
        m->A = materials[5 * i + 1];
        m->rho = materials[5 * i + 2];
        m->I_eV = materials[5 * i + 3];
        m->bk = materials[5 * i + 4];
        m->vacuum = !(m->rho > 0.0);
        if (!m->vacuum) {
            m->n_at = m->rho * NAVO / m->A;
            m->n_el = m->Z * m->n_at;
            m->x0_cm = orc_x0_gcm2(m->Z, m->A) / m->rho;
        }
    }
    h->cut[0] = physics[0];
    h->cut[1] = physics[1];
    h->cut[2] = physics[2];
    h->e_lo = physics[3];
    h->e_hi = physics[4];
    h->bpd = (int)physics[5];
    h->step_frac = physics[6];
    h->final_range = physics[7];
    h->mask = (unsigned)physics[8];
    h->n_grid = (int)floor(h->bpd * log10(h->e_hi / h->e_lo) + 0.5) + 1;
    h->grid = (double*)malloc(sizeof(double) * h->n_grid);
    h->igrid = (double*)calloc((size_t)h->n_grid, sizeof(double));
    h->irs = (double*)calloc((size_t)(n_mat > 0 ? n_mat : 1) * 3 * h->n_grid, sizeof(double));
    h->table = (double*)calloc((size_t)(n_mat > 0 ? n_mat : 1) * 3 * NQ * h->n_grid, sizeof(double));
    h->n_layers = n_layers;
    h->zb[0] = world[0];
    for (int i = 0; i < n_layers; ++i) {
        h->layer_mat[i] = (int)layers[3 * i + 0];
        h->zb[i + 1] = h->zb[i] + layers[3 * i + 1];
        h->layer_bin[i] = (int)layers[3 * i + 2];
    }
    h->hx = world[1];
    h->hy = world[2];
    for (int a = 0; a < 3; ++a) {
        h->wlo[a] = world[3 + a];
        h->whi[a] = world[6 + a];
        h->B[a] = world[9 + a];
    }
    h->rk_delta = world[12];
    h->max_steps = (int)world[13];
    h->n_bins = (int)world[14];
    h->max_field_step = world[15];
    h->has_field = (h->B[0] != 0.0 || h->B[1] != 0.0 || h->B[2] != 0.0);
    h->geom = (int)world[16];
    h->half_z = world[17];
    h->score_z = (int)world[18];
    h->zs_lo = world[19];
    h->zs_scale = (double)h->n_bins / (world[20] - world[19]);
    if ((h->geom != 0 && h->geom != 1) || (h->geom == 1 && (h->zb[0] != 0.0 || !(h->half_z > 0.0))) ||
        (h->score_z && !(world[20] > world[19]))) {
        orc_destroy(h);
        return NULL;
    }
    h->seed = seed;
    build_tables(h);
    return h;
}

void orc_destroy(orc_handle* h)
{
    if (!h) return;
    free(h->grid);
    free(h->igrid);
    free(h->irs);
    free(h->table);
    free(h);
}

int orc_grid_size(const orc_handle* h) { return h->n_grid; }

int orc_get_table(const orc_handle* h, int m, int p, int q, double* out)
{
    if (m < 0 || m >= h->n_mat || p < 0 || p > 2 || q < 0 || q > 5) return -1;
    const double* src = q == 5 ? h->grid : tab(h, m, p, q);
    memcpy(out, src, sizeof(double) * h->n_grid);
    return h->n_grid;
}

/* ------------------------------------------------------------------ */
/* Geometry (a reading of Sec. 2.3: the paper navigates CMS with       */
/* VecGeom or ORANGE, a CSG of quadric surfaces; here two simple kinds */
/* of volumes with exact logical volume indices).                      */
/* Layers: slabs stacked along +z from z0 inside |x|<=hx, |y|<=hy;     */
/* volume -1 is the vacuum of the world box; -2 is outside the world.  */
/* Cylinders: concentric shells about the z axis (Sec. 3.2's test        */
/* problem), shell i spanning zb[i] <= rho < zb[i+1] and |z| <= half_z,*/
/* zb[0] = 0; leaving the outermost shell or the end planes leaves the */
/* world (-2).                                                         */
/* ------------------------------------------------------------------ */
#define VOL_WORLD (-1)
#define VOL_OUT (-2)
#define GEOM_LAYERS 0
#define GEOM_CYLINDERS 1

typedef struct {
    double t;
    int next;
    int axis;
    double plane;
} exit_t;

/* locate the layer containing z on the stack (for entries through side
 * faces): largest j with zb[j] <= z, clamped to [0, n_layers-1] */
static int layer_at(const orc_handle* h, double z)
{
    int j = 0;
    while (j + 1 < h->n_layers && h->zb[j + 1] <= z) ++j;
    return j;
}

/* Cylinders: exit parameter along d (any length) from p in shell vol.
 * Candidates in the order end plane, outer surface, inner surface; the
 * smallest wins, ties to the earlier.  A surface rho = r meets the line
 * p + t d where a t^2 + 2 b t + c = 0, with a = dx^2 + dy^2,
 * b = px dx + py dy, c = px^2 + py^2 - r^2.  Outer surface (c <= 0): the
 * larger root, (sqrt(b^2 - a c) - b)/a, written -c/(b + sqrt(b^2 - a c))
 * when b > 0 to avoid cancellation.  Inner surface: only when moving
 * inward (b < 0) and the discriminant is non-negative, the smaller root
 * c/(sqrt(b^2 - a c) - b).  Crossing a radial surface moves the track to
 * the neighbouring shell; the end planes and the outermost surface lead
 * out of the world. */
static exit_t nav_exit_cyl(const orc_handle* h, int vol, const double p[3], const double d[3])
{
    exit_t e = {INF_D, VOL_OUT, -1, 0.0};
    if (d[2] != 0.0) {
        double pl = d[2] > 0.0 ? h->half_z : -h->half_z;
        e.t = (pl - p[2]) / d[2];
        e.axis = 2;
        e.plane = pl;
    }
    double a = d[0] * d[0] + d[1] * d[1];
    if (a > 0.0) {
        double b = p[0] * d[0] + p[1] * d[1];
        double q = p[0] * p[0] + p[1] * p[1];
        double ro = h->zb[vol + 1];
        double c = q - ro * ro;
        double disc = b * b - a * c;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double t = b > 0.0 ? -c / (b + sq) : (sq - b) / a;
        if (t < e.t) {
            e.t = t;
            e.axis = -1;
            e.plane = 0.0;
            e.next = vol + 1 < h->n_layers ? vol + 1 : VOL_OUT;
        }
        if (vol > 0 && b < 0.0) {
            double ri = h->zb[vol];
            double ci = q - ri * ri;
            double di = b * b - a * ci;
            if (di >= 0.0) {
                double ti = ci / (sqrt(di) - b);
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

/* exit parameter t >= 0 along d (any length) from point p in volume vol */
static exit_t nav_exit(const orc_handle* h, int vol, const double p[3], const double d[3])
{
    if (h->geom == GEOM_CYLINDERS) return nav_exit_cyl(h, vol, p, d);
    exit_t e = {INF_D, VOL_OUT, -1, 0.0};
    if (vol >= 0) {
        int L = h->n_layers;
        if (d[2] > 0.0) {
            double t = (h->zb[vol + 1] - p[2]) / d[2];
            if (t < e.t) {
                e.t = t;
                e.next = vol + 1 < L ? vol + 1 : VOL_WORLD;
                e.axis = 2;
                e.plane = h->zb[vol + 1];
            }
        } else if (d[2] < 0.0) {
            double t = (h->zb[vol] - p[2]) / d[2];
            if (t < e.t) {
                e.t = t;
                e.next = vol > 0 ? vol - 1 : VOL_WORLD;
                e.axis = 2;
                e.plane = h->zb[vol];
            }
        }
        double half[2] = {h->hx, h->hy};
        for (int a = 0; a < 2; ++a) {
            if (d[a] == 0.0) continue;
            double pl = d[a] > 0.0 ? half[a] : -half[a];
            double t = (pl - p[a]) / d[a];
            if (t < e.t) {
                e.t = t;
                e.next = VOL_WORLD;
                e.axis = a;
                e.plane = pl;
            }
        }
    } else {
        double lo[3] = {-h->hx, -h->hy, h->zb[0]};
        double hi[3] = {h->hx, h->hy, h->zb[h->n_layers]};
        static const int order[3] = {2, 0, 1};
        for (int oi = 0; oi < 3; ++oi) {
            int a = order[oi];
            if (d[a] == 0.0) continue;
            double pl = d[a] > 0.0 ? lo[a] : hi[a];
            double t = (pl - p[a]) / d[a];
            if (!(t >= 0.0) || !(t < e.t)) continue;
            int ok = 1;
            double q[3];
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                q[b] = p[b] + t * d[b];
                if (q[b] < lo[b] || q[b] > hi[b]) ok = 0;
            }
            if (!ok) continue;
            e.t = t;
            e.axis = a;
            e.plane = pl;
            if (a == 2)
                e.next = d[2] > 0.0 ? 0 : h->n_layers - 1;
            else
                e.next = layer_at(h, q[2]);
        }
        for (int oi = 0; oi < 3; ++oi) {
            int a = order[oi];
            if (d[a] == 0.0) continue;
            double pl = d[a] > 0.0 ? h->whi[a] : h->wlo[a];
            double t = (pl - p[a]) / d[a];
            if (t < e.t) {
                e.t = t;
                e.next = VOL_OUT;
                e.axis = a;
                e.plane = pl;
            }
        }
    }
    if (e.t < 0.0) e.t = 0.0;
    return e;
}

/* logical volume of a starting point (primaries) */
static int locate(const orc_handle* h, const double p[3])
{
    if (h->geom == GEOM_CYLINDERS) {
        double q = p[0] * p[0] + p[1] * p[1];
        double rmax = h->zb[h->n_layers];
        if (!(p[2] >= -h->half_z && p[2] <= h->half_z) || !(q < rmax * rmax)) return VOL_OUT;
        int j = 0;
        while (j + 1 < h->n_layers && h->zb[j + 1] * h->zb[j + 1] <= q) ++j;
        return j;
    }
    if (p[0] >= -h->hx && p[0] <= h->hx && p[1] >= -h->hy && p[1] <= h->hy && p[2] >= h->zb[0] &&
        p[2] <= h->zb[h->n_layers])
        return layer_at(h, p[2]);
    for (int a = 0; a < 3; ++a)
        if (p[a] < h->wlo[a] || p[a] > h->whi[a]) return VOL_OUT;
    return VOL_WORLD;
}

/* ------------------------------------------------------------------ */
/* Direction helpers                                                   */
/* ------------------------------------------------------------------ */
/* rotate the local direction (sin t cos phi, sin t sin phi, cos t),
 * given in the frame whose z axis is u, into the global frame */
static void rotate(const double u[3], double cost, double phi, double out[3])
{
    double sint = sqrt(fmax(0.0, (1.0 - cost) * (1.0 + cost)));
    double a = sint * cos(phi);
    double b = sint * sin(phi);
    double perp2 = u[0] * u[0] + u[1] * u[1];
    if (perp2 > 1e-20) {
        double up = sqrt(perp2);
        out[0] = (u[0] * u[2] * a - u[1] * b) / up + u[0] * cost;
        out[1] = (u[1] * u[2] * a + u[0] * b) / up + u[1] * cost;
        out[2] = -up * a + u[2] * cost;
    } else if (u[2] >= 0.0) {
        out[0] = a;
        out[1] = b;
        out[2] = cost;
    } else {
        out[0] = -a;
        out[1] = b;
        out[2] = -cost;
    }
}

/* out = normalize(pa*da - pb*db); returns 0 if the difference vanishes */
static int momentum_balance(double pa, const double da[3], double pb, const double db[3], double out[3])
{
    double v0 = pa * da[0] - pb * db[0];
    double v1 = pa * da[1] - pb * db[1];
    double v2 = pa * da[2] - pb * db[2];
    double n = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    if (!(n > 0.0)) return 0;
    out[0] = v0 / n;
    out[1] = v1 / n;
    out[2] = v2 / n;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Interaction samplers (draws 2, 3, ... of the step, in program order) */
/* Each writes products: sec_t[k] (type), sec_T[k], sec_dir[k][3].     */
/* The parent's new energy/direction is returned through *T, dir.      */
/* ------------------------------------------------------------------ */
enum { P_PHOTO = 0, P_COMPTON = 1, P_PAIR = 2, P_IONI = 3, P_BREMS = 4, P_ANNIH = 5, P_RAYLEIGH = 9 };

/* Every rejection loop accepts its candidate after MAX_TRIALS trials (a
 * safety bound against non-finite input; every acceptance probability here
 * is at least 1/3, so a valid input never reaches it). */
#define MAX_TRIALS 1000

typedef struct {
    int n;
    int type[2];
    double T[2];
    double dir[2][3];
    double local; /* energy deposited locally by the interaction itself */
    int parent_alive;
    int null_interaction;
} products_t;

/* Compton, Klein-Nishina: composition of 1/eps and eps densities on
 * [eps0, 1], eps0 = 1/(1+2 kappa), weights ln(1/eps0) and (1-eps0^2)/2,
 * rejection with g = 1 - eps sin^2/(1+eps^2) (Butcher & Messel, Nucl.
 * Phys. 20 (1960) 15).  Free electron at rest (no binding, no Doppler). */
static void sample_compton(draws_t* d, double k, double dir[3], products_t* out, double* knew)
{
    double kappa = k / ME;
    double eps0 = 1.0 / (1.0 + 2.0 * kappa);
    double eps0sq = eps0 * eps0;
    double a1 = -log(eps0);
    double a2 = 0.5 * (1.0 - eps0sq);
    double eps, epssq, onecost, sint2, g;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d), u3 = draw(d);
        if (a1 / (a1 + a2) > u1) {
            eps = exp(-a1 * u2);
            epssq = eps * eps;
        } else {
            epssq = eps0sq + (1.0 - eps0sq) * u2;
            eps = sqrt(epssq);
        }
        onecost = (1.0 - eps) / (eps * kappa);
        sint2 = onecost * (2.0 - onecost);
        g = 1.0 - eps * sint2 / (1.0 + epssq);
        if (u3 <= g || trial >= MAX_TRIALS) break;
    }
    double phi = 2.0 * PI * draw(d);
    double cost = 1.0 - onecost;
    double kp = eps * k;
    double gdir[3];
    rotate(dir, cost, phi, gdir);
    out->n = 0;
    double Te = k - kp;
    double edir[3];
    if (Te > 0.0 && momentum_balance(k, dir, kp, gdir, edir)) {
        out->type[0] = 1;
        out->T[0] = Te;
        memcpy(out->dir[0], edir, sizeof edir);
        out->n = 1;
    } else {
        out->local += Te;
    }
    memcpy(dir, gdir, sizeof gdir);
    *knew = kp;
    out->parent_alive = 1;
}

/* Bethe-Heitler (complete screening): x uniform on [eps0, 1-eps0],
 * accept with 1 - 4/3 x(1-x) (<= 1).  Both leptons along the photon. */
/* Rayleigh angle: x = 1 - cos(theta) from (1 + b x)^-4 by inversion,
 * (1 + b x)^-3 = 1 - u (1 - (1 + 2b)^-3) (written with log1p/expm1,
 * exact for small b), accepted with (1 + (1 - x)^2)/2; the photon keeps its
 * energy; azimuth 2 pi u. */
static void sample_rayleigh(draws_t* d, double k, double Z, double dir[3])
{
    double b = rayleigh_b(Z, k);
    double tail = -expm1(-3.0 * log1p(2.0 * b));
    double x;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        x = expm1(-log1p(-u1 * tail) / 3.0) / b;
        if (x > 2.0) x = 2.0;
        if (2.0 * u2 <= 2.0 - 2.0 * x + x * x || trial >= MAX_TRIALS) break;
    }
    double phi = 2.0 * PI * draw(d);
    double out[3];
    double cost = 1.0 - x;
    rotate(dir, cost, phi, out);
    memcpy(dir, out, sizeof out);
}

/* Photoelectron angle (angular option): Sauter's K-shell distribution,
 * dN/dcos ~ sin^2(theta) / (1 - beta cos)^4 [1 + g (1 - beta cos)],
 * g = gamma (gamma - 1) (gamma - 2) / 2.  In v = 1 - beta cos, v in
 * [a, 2 - a] (a = 1 - beta), the density is f(v) = (v - a)(2 - a - v)
 * (1 + g v) / v^4, bounded by 16 [(v + a)^-3 + max(g, 0) (v + a)^-2];
 * both envelope terms invert in closed form.  Returns 1 - cos(theta) =
 * (v - a)/beta.  Below beta = 1e-3 the direction is isotropic. */
static double sauter_one_minus_cos(draws_t* d, double T)
{
    double E = T + ME;
    double p = sqrt(T * (T + 2.0 * ME));
    double beta = p / E;
    if (!(beta > 1e-3)) return 2.0 * draw(d);
    double gam = E / ME;
    double a = ME * ME / (E * (E + p));
    double g = 0.5 * gam * (gam - 1.0) * (gam - 2.0);
    double gp = g > 0.0 ? g : 0.0;
    double i2a = 1.0 / (2.0 * a);
    double w1 = 0.5 * (i2a * i2a - 0.25), w2 = gp * (i2a - 0.5);
    double v = a;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d), u3 = draw(d);
        if (u1 * (w1 + w2) < w1) {
            double w = i2a * i2a * (1.0 - u2) + 0.25 * u2; /* (v + a)^-2 */
            v = 1.0 / sqrt(w) - a;
        } else {
            double w = i2a * (1.0 - u2) + 0.5 * u2; /* (v + a)^-1 */
            v = 1.0 / w - a;
        }
        double va = v + a;
        double f = (v - a) * (2.0 - a - v) * (1.0 + g * v) / (v * v * v * v);
        double env = 16.0 * (1.0 / (va * va * va) + gp / (va * va));
        if (u3 * env <= f || trial >= MAX_TRIALS) break;
    }
    return (v - a) / beta;
}

/* Angular distribution of a lepton or photon emitted by a lepton of
 * kinetic energy T (angular option, process bit ORC_ANGULAR): the dipole
 * form dN/dcos(theta) ~ (1 - beta cos(theta))^-2, whose width is ~1/gamma
 * (the leading behaviour of the Sauter and Schiff distributions).
 * Inverting its cumulative distribution at u gives, with a = 1 - beta,
 * 1 - cos(theta) = 2 a (1 - u) / (a + 2 beta u), free of cancellation as
 * beta -> 1 (a = me^2 / (E (E + p)) computed directly). */
static double dipole_one_minus_cos(double T, double u)
{
    double E = T + ME;
    double p = sqrt(T * (T + 2.0 * ME));
    double beta = p / E;
    double a = ME * ME / (E * (E + p));
    return 2.0 * a * (1.0 - u) / (a + 2.0 * beta * u);
}

/* direction at polar angle theta (1 - cos given) and azimuth phi about dir */
static void emit_dir(const double dir[3], double omc, double phi, double out[3])
{
    double cost = 1.0 - omc;
    if (cost < -1.0) cost = -1.0;
    rotate(dir, cost, phi, out);
}

static void sample_pair(draws_t* d, double k, const double dir[3], products_t* out, int angular)
{
    double eps0 = ME / k;
    double w = 1.0 - 2.0 * eps0;
    double x;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        x = eps0 + w * u1;
        double f = 1.0 - 4.0 / 3.0 * x * (1.0 - x);
        if (u2 <= f || trial >= MAX_TRIALS) break;
    }
    double Tm = x * k - ME;
    if (Tm < 0.0) Tm = 0.0;
    double Tp = (k - Tm) - 2.0 * ME;
    if (Tp < 0.0) Tp = 0.0;
    out->n = 2;
    out->type[0] = 1;
    out->T[0] = Tm;
    out->type[1] = 2;
    out->T[1] = Tp;
    if (angular) {
        /* each lepton at its own dipole angle; azimuths phi and phi + pi */
        double um = draw(d), phi = 2.0 * PI * draw(d), up = draw(d);
        emit_dir(dir, dipole_one_minus_cos(Tm, um), phi, out->dir[0]);
        emit_dir(dir, dipole_one_minus_cos(Tp, up), phi + PI, out->dir[1]);
    } else {
        for (int a = 0; a < 3; ++a) {
            out->dir[0][a] = dir[a];
            out->dir[1][a] = dir[a];
        }
    }
    out->parent_alive = 0;
}

/* photoelectric stand-in: photoelectron T = k - bk along the photon,
 * binding energy bk deposited locally */
static void sample_photo(draws_t* d, double k, double bk, const double dir[3], products_t* out, int angular)
{
    out->n = 1;
    out->type[0] = 1;
    out->T[0] = k - bk;
    if (angular) {
        double omc = sauter_one_minus_cos(d, k - bk);
        double phi = 2.0 * PI * draw(d);
        emit_dir(dir, omc, phi, out->dir[0]);
    } else {
        for (int a = 0; a < 3; ++a) out->dir[0][a] = dir[a];
    }
    out->local += bk;
    out->parent_alive = 0;
}

/* bremsstrahlung: k = kc (T/kc)^u (1/k envelope), accept with
 * (4/3 - 4/3 y + y^2)/(4/3); photon along the lepton */
static void sample_brems(draws_t* d, double T, double kc, const double dir[3], products_t* out, double* Tnew,
                         int angular)
{
    double E = T + ME;
    double lr = log(T / kc);
    double k;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        k = kc * exp(u1 * lr);
        double y = k / E;
        double f = 4.0 / 3.0 - 4.0 / 3.0 * y + y * y;
        if (u2 * (4.0 / 3.0) <= f || trial >= MAX_TRIALS) break;
    }
    out->n = 1;
    out->type[0] = 0;
    out->T[0] = k;
    if (angular) {
        /* photon at the dipole angle of the radiating lepton; the lepton
         * keeps its direction (the nucleus takes the recoil) */
        double u = draw(d), phi = 2.0 * PI * draw(d);
        emit_dir(dir, dipole_one_minus_cos(T, u), phi, out->dir[0]);
    } else {
        for (int a = 0; a < 3; ++a) out->dir[0][a] = dir[a];
    }
    *Tnew = T - k;
    out->parent_alive = 1;
}

/* delta-ray kinematics shared by Moller and Bhabha: delta at
 * cos = sqrt(Td (T+2me) / (T (Td+2me))), parent from momentum balance */
static void delta_kinematics(draws_t* d, double T, double Td, double dir[3], products_t* out, double* Tnew)
{
    double cost = sqrt(Td * (T + 2.0 * ME) / (T * (Td + 2.0 * ME)));
    if (cost > 1.0) cost = 1.0;
    double phi = 2.0 * PI * draw(d);
    double ddir[3];
    rotate(dir, cost, phi, ddir);
    double p0 = sqrt(T * (T + 2.0 * ME));
    double pd = sqrt(Td * (Td + 2.0 * ME));
    double ndir[3];
    if (momentum_balance(p0, dir, pd, ddir, ndir)) memcpy(dir, ndir, sizeof ndir);
    out->n = 1;
    out->type[0] = 1;
    out->T[0] = Td;
    memcpy(out->dir[0], ddir, sizeof ddir);
    *Tnew = T - Td;
    out->parent_alive = 1;
}

/* Moller: eps = xc / (1 - u (1 - 2 xc)) (1/eps^2 envelope on [xc,1/2]),
 * accept with eps^2 B(eps) / (2 + g1^2/4) */
static void sample_moller(draws_t* d, double T, double cut, double dir[3], products_t* out, double* Tnew)
{
    double xc = cut / T;
    double g = (T + ME) / ME;
    double g1 = (g - 1.0) / g;
    double c = (2.0 * g - 1.0) / (g * g);
    double gmax = 2.0 + 0.25 * g1 * g1;
    double eps;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        eps = xc / (1.0 - u1 * (1.0 - 2.0 * xc));
        double q = eps / (1.0 - eps);
        double f = 1.0 + q * q + g1 * g1 * eps * eps - c * q;
        if (u2 * gmax <= f || trial >= MAX_TRIALS) break;
    }
    delta_kinematics(d, T, eps * T, dir, out, Tnew);
}

/* Bhabha: eps = xc / (1 - u (1 - xc)) (1/eps^2 envelope on [xc,1]),
 * accept with beta^2 eps^2 (dsigma/deps bracket) (<= 1) */
static void sample_bhabha(draws_t* d, double T, double cut, double dir[3], products_t* out, double* Tnew)
{
    double xc = cut / T;
    double b2, c1, c2, c3, c4;
    bhabha_coeffs(T, &b2, &c1, &c2, &c3, &c4);
    double eps;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        eps = xc / (1.0 - u1 * (1.0 - xc));
        double f = 1.0 - b2 * eps * (c1 - eps * (c2 - eps * (c3 - eps * c4)));
        if (u2 <= f || trial >= MAX_TRIALS) break;
    }
    delta_kinematics(d, T, eps * T, dir, out, Tnew);
}

/* annihilation in flight: eps = emin (emax/emin)^u (1/eps envelope),
 * accept with eps S(eps)/(g^2+4g+1) = 1 - ((g+1)^2 eps + 1/eps)/(g^2+4g+1).
 * Photon 1 at cos = (T+2me)(E1-me)/(p E1), photon 2 by momentum balance. */
static void sample_annih(draws_t* d, double T, const double dir[3], products_t* out)
{
    double tau = T / ME;
    double g = tau + 1.0;
    double a = tau + 2.0;
    double s = sqrt(tau * (tau + 2.0));
    double emin = 0.5 * (1.0 - s / a);
    double emax = 1.0 - emin;
    double lr = log(emax / emin);
    double bq = g * g + 4.0 * g + 1.0;
    double eps;
    for (int trial = 1;; ++trial) {
        double u1 = draw(d), u2 = draw(d);
        eps = emin * exp(u1 * lr);
        double f = 1.0 - (a * a * eps + 1.0 / eps) / bq;
        if (u2 <= f || trial >= MAX_TRIALS) break;
    }
    double Etot = T + 2.0 * ME;
    double E1 = eps * Etot;
    double E2 = Etot - E1;
    double p = sqrt(T * (T + 2.0 * ME));
    double cost = Etot * (E1 - ME) / (p * E1);
    if (cost > 1.0) cost = 1.0;
    if (cost < -1.0) cost = -1.0;
    double phi = 2.0 * PI * draw(d);
    double d1[3], d2[3];
    rotate(dir, cost, phi, d1);
    if (!momentum_balance(p, dir, E1, d1, d2)) {
        d2[0] = -d1[0];
        d2[1] = -d1[1];
        d2[2] = -d1[2];
    }
    out->n = 2;
    out->type[0] = 0;
    out->T[0] = E1;
    memcpy(out->dir[0], d1, sizeof d1);
    out->type[1] = 0;
    out->T[1] = E2;
    memcpy(out->dir[1], d2, sizeof d2);
    out->parent_alive = 0;
}

/* single-interaction sampler entry for brute-force histogram pins.
 * out: {parent E after, parent dir[3], n, (type, T, dir[3]) x 2, local} */
int orc_sample(int process, double E, double cut_e, double cut_g, uint32_t seed, uint64_t event_id,
               uint64_t uid, uint32_t step, double* out)
{
    draws_t dr = {seed, event_id, uid, step, 2};
    double dir[3] = {0.0, 0.0, 1.0};
    products_t pr;
    memset(&pr, 0, sizeof pr);
    double Enew = E;
    switch (process) {
    case P_PHOTO: sample_photo(&dr, E, cut_e, dir, &pr, 0); Enew = 0.0; break;
    case 10: sample_photo(&dr, E, cut_e, dir, &pr, 1); Enew = 0.0; break;
    case P_RAYLEIGH: sample_rayleigh(&dr, E, cut_e, dir); break; /* cut_e carries Z */
    case P_COMPTON: sample_compton(&dr, E, dir, &pr, &Enew); break;
    case P_PAIR: sample_pair(&dr, E, dir, &pr, 0); Enew = 0.0; break;
    case 8: sample_pair(&dr, E, dir, &pr, 1); Enew = 0.0; break;
    case P_IONI: sample_moller(&dr, E, cut_e, dir, &pr, &Enew); break;
    case P_BREMS: sample_brems(&dr, E, cut_g, dir, &pr, &Enew, 0); break;
    case 7: sample_brems(&dr, E, cut_g, dir, &pr, &Enew, 1); break;
    case P_ANNIH: sample_annih(&dr, E, dir, &pr); Enew = 0.0; break;
    case 6: sample_bhabha(&dr, E, cut_e, dir, &pr, &Enew); break;
    default: return -1;
    }
    out[0] = Enew;
    out[1] = dir[0];
    out[2] = dir[1];
    out[3] = dir[2];
    out[4] = pr.n;
    for (int k = 0; k < 2; ++k) {
        out[5 + 5 * k] = k < pr.n ? pr.type[k] : -1;
        out[6 + 5 * k] = k < pr.n ? pr.T[k] : 0.0;
        for (int a = 0; a < 3; ++a) out[7 + 5 * k + a] = k < pr.n ? pr.dir[k][a] : 0.0;
    }
    out[15] = pr.local;
    return (int)dr.next;
}

/* ------------------------------------------------------------------ */
/* Field propagation: classical RK4 in path length on (x, u) with      */
/* du/ds = q (c/p) u x B, |p| fixed during the step; substep           */
/* h <= sqrt(8 r delta) (sagitta <= delta); after each substep the     */
/* chord is tested against the current volume, and a crossing at chord */
/* fraction f repeats the substep with h f and snaps onto the plane.   */
/* (Sec. 2.3 says only that propagation is on-device with selectable   */
/* integrators; this is a reading.)                                    */
/* ------------------------------------------------------------------ */
/* A step in a field is a whole number n of equal RK4 substeps of at most
 * h_max: n = ceil(s / h_max) substeps of s / n for a step limit s up to
 * MAX_SUBSTEPS h_max (and up to max_field_step).  A longer step is cut to
 * exactly MAX_SUBSTEPS substeps of h_max and ends without an interaction;
 * the track continues at its next step (a reading: it bounds the work of
 * one step of a looping low-energy track).  The cut step's substep count
 * is set, not recomputed from s / h_max, whose rounding would otherwise
 * decide between MAX_SUBSTEPS and MAX_SUBSTEPS + 1 substeps. */
#define MAX_SUBSTEPS 100

/* The RK4 arithmetic is written with fused multiply-adds where a product
 * is added (one rounding each; a reading: the integrator's rounding is not
 * fixed by the paper). */
static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = fma(a[1], b[2], -(a[2] * b[1]));
    o[1] = fma(a[2], b[0], -(a[0] * b[2]));
    o[2] = fma(a[0], b[1], -(a[1] * b[0]));
}

static void rk4(const orc_handle* h, double kq, const double x[3], const double u[3], double hs, double xo[3],
                double uo[3])
{
    double a1[3], a2[3], a3[3], a4[3], u2[3], u3[3], u4[3], t[3];
    double hh = 0.5 * hs;
    cross(u, h->B, t);
    for (int i = 0; i < 3; ++i) a1[i] = kq * t[i];
    for (int i = 0; i < 3; ++i) u2[i] = fma(hh, a1[i], u[i]);
    cross(u2, h->B, t);
    for (int i = 0; i < 3; ++i) a2[i] = kq * t[i];
    for (int i = 0; i < 3; ++i) u3[i] = fma(hh, a2[i], u[i]);
    cross(u3, h->B, t);
    for (int i = 0; i < 3; ++i) a3[i] = kq * t[i];
    for (int i = 0; i < 3; ++i) u4[i] = fma(hs, a3[i], u[i]);
    cross(u4, h->B, t);
    for (int i = 0; i < 3; ++i) a4[i] = kq * t[i];
    double h6 = hs / 6.0;
    for (int i = 0; i < 3; ++i) {
        double su = fma(2.0, u3[i], fma(2.0, u2[i], u[i])) + u4[i];
        double sa = fma(2.0, a3[i], fma(2.0, a2[i], a1[i])) + a4[i];
        xo[i] = fma(h6, su, x[i]);
        uo[i] = fma(h6, sa, u[i]);
    }
    double n = sqrt(fma(uo[0], uo[0], fma(uo[1], uo[1], uo[2] * uo[2])));
    for (int i = 0; i < 3; ++i) uo[i] = uo[i] / n;
}

/* propagate a charged track along the field by n substeps of length hs
 * (or up to the first boundary crossing); returns the path length;
 * *bnd receives the crossing */
static double propagate_field(const orc_handle* h, int charge, double T, int vol, double x[3], double u[3],
                              int n, double hs, exit_t* bnd, int* crossed)
{
    double p = sqrt(T * (T + 2.0 * ME));
    double kq = charge * FIELD_C / p;
    double s = 0.0;
    *crossed = 0;
    for (int i = 0; i < n; ++i) {
        double x1[3], u1[3], c[3];
        rk4(h, kq, x, u, hs, x1, u1);
        for (int a = 0; a < 3; ++a) c[a] = x1[a] - x[a];
        exit_t e = nav_exit(h, vol, x, c);
        if (e.t <= 1.0) {
            double h2 = hs * e.t;
            rk4(h, kq, x, u, h2, x1, u1);
            if (e.axis >= 0) x1[e.axis] = e.plane;
            memcpy(x, x1, sizeof x1);
            memcpy(u, u1, sizeof u1);
            s += h2;
            *bnd = e;
            *crossed = 1;
            return s;
        }
        memcpy(x, x1, sizeof x1);
        memcpy(u, u1, sizeof u1);
        s += hs;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Transport                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int type; /* 0 gamma, 1 e-, 2 e+ */
    double T;
    double x[3], u[3];
    int vol;
    uint64_t uid;
    uint32_t step;
} track_t;

typedef struct {
    double* hist;
    double edep, escaped, killed, e_in;
    double n_steps, n_tracks;
} tally_t;

/* histogram bin of a deposit made in volume vol at height z: the
 * volume's score bin, or with scoring along z the bin of z among n_bins
 * equal bins of [zs_lo, zs_hi), floor((z - zs_lo) * n_bins / (zs_hi -
 * zs_lo)) with the scale factor rounded once; -1 = no bin (the deposit still counts in
 * edep) */
static int score_bin(const orc_handle* h, int vol, double z)
{
    if (h->score_z) {
        double f = floor((z - h->zs_lo) * h->zs_scale);
        return (f >= 0.0 && f < (double)h->n_bins) ? (int)f : -1;
    }
    if (vol < 0) return -1;
    int b = h->layer_bin[vol];
    return (b >= 0 && b < h->n_bins) ? b : -1;
}

/* every deposit of a step is made at the post-step point, in the volume
 * the step started in */
static void deposit(const orc_handle* h, tally_t* t, int vol, double z, double e)
{
    t->edep += e;
    int b = score_bin(h, vol, z);
    if (b >= 0) t->hist[b] += e;
}

static double rest_energy(int type) { return type == 2 ? 2.0 * ME : 0.0; }

/* ------------------------------------------------------------------ */
/* Multiple scattering of e+- (process bit ORC_MSC; Table 1 lists Urban */
/* and WentzelVI, whose data and tuned parameters are not available).  */
/* A reading with a published closed form: after a step of length s in */
/* matter the direction turns by a polar angle whose two projections   */
/* are independent Gaussians of width theta0 from Highland's formula    */
/* (PDG review "Passage of particles through matter", Eq. 34.15, unit  */
/* charge): theta0 = 13.6 MeV / (beta p) sqrt(s/X0) [1 + 0.038         */
/* ln(s / (X0 beta^2))], with the pre-step momentum, clamped at 0 where */
/* the bracket turns negative (s/X0 < 1e-11).  The space angle is then */
/* theta = theta0 sqrt(-2 ln u_a), the azimuth 2 pi u_b (u_a, u_b: the  */
/* step's draws MSC_DRAW, MSC_DRAW + 1), capped at pi.  No lateral     */
/* displacement and no path-length correction.                         */
/* ------------------------------------------------------------------ */
#define MSC_DRAW (1u << 20)

double orc_highland(double T, double s, double x0_cm)
{
    double p = sqrt(T * (T + 2.0 * ME));
    double beta = p / (T + ME);
    double t = s / x0_cm;
    double f = 1.0 + 0.038 * log(t / (beta * beta));
    if (!(f > 0.0)) return 0.0;
    return 13.6 / (beta * p) * sqrt(t) * f;
}

static void msc_deflect(draws_t* d, double T, double s, double x0_cm, double u[3])
{
    double th0 = orc_highland(T, s, x0_cm);
    if (!(th0 > 0.0)) return;
    d->next = MSC_DRAW;
    double ua = draw(d), ub = draw(d);
    double th = th0 * sqrt(-2.0 * log(ua));
    if (th > PI) th = PI;
    double out[3];
    rotate(u, cos(th), 2.0 * PI * ub, out);
    memcpy(u, out, sizeof out);
}

int orc_msc(double T, double s, double x0_cm, uint32_t seed, uint64_t event_id, uint64_t uid, uint32_t step,
            double* dir)
{
    draws_t dr = {seed, event_id, uid, step, 0};
    msc_deflect(&dr, T, s, x0_cm, dir);
    return (int)dr.next;
}

typedef struct {
    double s, edep;
    int boundary, interacted, process, alive, msc;
    int n_sec;
    track_t sec[2];
} step_result_t;

/* One step of one track, in the order documented in the module notes:
 *  1. cross sections at the pre-step energy (vacuum: none)
 *  2. s_int = -ln(u0)/Sigma_tot                        (draw 0)
 *  3. e+-: s_max = max(step_frac R, min(R, final_range))
 *  4. s_phys = min(s_int, s_max); field steps also <= max_field_step
 *  5. propagate (straight or RK4) to min(s_phys, boundary); ties -> boundary
 *  6. e+-: T' = R^-1(R(T) - s), deposit T - T' in the volume traversed
 *  7. e+- below cut: deposit T' (+2me for e+), track ends
 *  8. boundary: logical volume update; leaving the world tallies escape
 *  9. interaction-limited: process by u1 * Sigma_tot against the
 *     cumulative pre-step Sigma's (draw 1), sampled with the post-loss T
 * 10. step += 1; at max_steps the track is killed                        */
static void step_track(const orc_handle* h, uint64_t event_id, track_t* tr, tally_t* ta, step_result_t* res)
{
    memset(res, 0, sizeof *res);
    res->process = -1;
    res->alive = 1;
    draws_t dr = {h->seed, event_id, tr->uid, tr->step, 0};
    int mi = tr->vol >= 0 ? h->layer_mat[tr->vol] : -1;
    const mat_t* m = (mi >= 0 && mi < h->n_mat && !h->mat[mi].vacuum) ? &h->mat[mi] : NULL;
    int charged = tr->type != 0;
    double sig[4] = {0.0, 0.0, 0.0, 0.0};
    /* photons: photo, Compton, pair (+ Rayleigh); e-: ioni, brems;
     * e+: ioni, brems, annihilation */
    int nproc = tr->type == 2 ? 3 : (tr->type == 1 ? 2 : ((h->mask & ORC_RAYLEIGH) ? 4 : 3));
    double sig_tot = 0.0;
    double R = 0.0;
    if (m) {
        for (int i = 0; i < nproc; ++i) sig[i] = lookup(h, tab(h, mi, tr->type, i), tr->T);
        sig_tot = sig[0] + sig[1];
        if (nproc >= 3) sig_tot = sig_tot + sig[2];
        if (nproc == 4) sig_tot = sig_tot + sig[3];
    }
    double s_int = INF_D;
    if (sig_tot > 0.0) {
        dr.next = 0;
        s_int = -log(draw(&dr)) / sig_tot;
    }
    double s_max = INF_D;
    if (charged && m) {
        R = range_of(h, tab(h, mi, tr->type, 3), tr->T);
        double lim = R < h->final_range ? R : h->final_range;
        double fr = h->step_frac * R;
        s_max = fr > lim ? fr : lim;
    }
    double s_phys = s_max;
    int interact = 0;
    if (s_int < s_max) {
        s_phys = s_int;
        interact = 1;
    }
    int use_field = charged && h->has_field;
    double s;
    int boundary = 0;
    exit_t e;
    if (!use_field) {
        e = nav_exit(h, tr->vol, tr->x, tr->u);
        if (e.t <= s_phys) {
            s = e.t;
            boundary = 1;
        } else {
            s = s_phys;
        }
        for (int a = 0; a < 3; ++a) tr->x[a] = fma(s, tr->u[a], tr->x[a]);
        if (boundary && e.axis >= 0) tr->x[e.axis] = e.plane;
    } else {
        double smax = s_phys;
        if (smax > h->max_field_step) {
            smax = h->max_field_step;
            interact = 0;
        }
        /* substeps of at most h_max = sqrt(8 r delta), r = p / (c |B|);
         * at most MAX_SUBSTEPS of them */
        double pm = sqrt(tr->T * (tr->T + 2.0 * ME));
        double bmag = sqrt(h->B[0] * h->B[0] + h->B[1] * h->B[1] + h->B[2] * h->B[2]);
        double hmax = sqrt(8.0 * (pm / (FIELD_C * bmag)) * h->rk_delta);
        int nsub;
        double hs;
        if (smax > MAX_SUBSTEPS * hmax) {
            nsub = MAX_SUBSTEPS;
            hs = hmax;
            interact = 0;
        } else {
            double ns = ceil(smax / hmax);
            if (ns < 1.0) ns = 1.0;
            nsub = (int)ns;
            hs = smax / ns;
        }
        int crossed = 0;
        s = propagate_field(h, tr->type == 1 ? -1 : 1, tr->T, tr->vol, tr->x, tr->u, nsub, hs, &e, &crossed);
        boundary = crossed;
        if (boundary) interact = 0;
    }
    if (boundary) interact = 0;
    res->s = s;
    res->boundary = boundary;
    int alive = 1;
    /* 6-7: continuous loss (and 6b: multiple scattering) */
    const double T0 = tr->T;
    if (charged && m) {
        double r = R - s;
        double Tn = r > 0.0 ? inv_range_of(h, tab(h, mi, tr->type, 3), irs_of(h, mi, tr->type), r) : 0.0;
        double ed = tr->T - Tn;
        deposit(h, ta, tr->vol, tr->x[2], ed);
        res->edep += ed;
        tr->T = Tn;
        if (tr->T < h->cut[tr->type]) {
            double e2 = tr->T + rest_energy(tr->type);
            deposit(h, ta, tr->vol, tr->x[2], e2);
            res->edep += e2;
            alive = 0;
        }
    }
    /* 6b: multiple scattering at the post-step point of a charged step in
     * matter (boundary steps included) */
    if (alive && charged && m && (h->mask & ORC_MSC) && s > 0.0) {
        msc_deflect(&dr, T0, s, m->x0_cm, tr->u);
        res->msc = 1;
    }
    /* 8: boundary */
    if (alive && boundary) {
        tr->vol = e.next;
        if (tr->vol == VOL_OUT) {
            ta->escaped += tr->T + rest_energy(tr->type);
            alive = 0;
        }
    } else if (alive && interact) {
        /* 9: select and sample */
        dr.next = 1;
        double x = draw(&dr) * sig_tot;
        int proc = nproc - 1;
        double c = 0.0;
        for (int i = 0; i < nproc; ++i) {
            c += sig[i];
            if (x < c) {
                proc = i;
                break;
            }
        }
        int pid; /* physics process id */
        if (tr->type == 0)
            pid = proc == 0 ? P_PHOTO : (proc == 1 ? P_COMPTON : (proc == 2 ? P_PAIR : P_RAYLEIGH));
        else
            pid = proc == 0 ? P_IONI : (proc == 1 ? P_BREMS : P_ANNIH);
        res->interacted = 1;
        res->process = pid;
        dr.next = 2;
        products_t pr;
        memset(&pr, 0, sizeof pr);
        pr.parent_alive = 1;
        double T = tr->T;
        double cut_e = h->cut[1], kc = h->cut[0];
        switch (pid) {
        case P_PHOTO:
            if (T > m->bk)
                sample_photo(&dr, T, m->bk, tr->u, &pr, (h->mask & ORC_ANGULAR) != 0);
            else
                pr.null_interaction = 1;
            break;
        case P_COMPTON: sample_compton(&dr, T, tr->u, &pr, &tr->T); break;
        case P_PAIR:
            if (T > 2.0 * ME)
                sample_pair(&dr, T, tr->u, &pr, (h->mask & ORC_ANGULAR) != 0);
            else
                pr.null_interaction = 1;
            break;
        case P_IONI:
            if (tr->type == 1) {
                if (T > 2.0 * cut_e)
                    sample_moller(&dr, T, cut_e, tr->u, &pr, &tr->T);
                else
                    pr.null_interaction = 1;
            } else {
                if (T > cut_e)
                    sample_bhabha(&dr, T, cut_e, tr->u, &pr, &tr->T);
                else
                    pr.null_interaction = 1;
            }
            break;
        case P_BREMS:
            if (T > kc)
                sample_brems(&dr, T, kc, tr->u, &pr, &tr->T, (h->mask & ORC_ANGULAR) != 0);
            else
                pr.null_interaction = 1;
            break;
        case P_ANNIH: sample_annih(&dr, T, tr->u, &pr); break;
        case P_RAYLEIGH: sample_rayleigh(&dr, T, m->Z, tr->u); break;
        }
        if (pr.local != 0.0) {
            deposit(h, ta, tr->vol, tr->x[2], pr.local);
            res->edep += pr.local;
        }
        for (int k = 0; k < pr.n; ++k) {
            int st = pr.type[k];
            double sT = pr.T[k];
            if (sT < h->cut[st]) {
                double e2 = sT + rest_energy(st);
                deposit(h, ta, tr->vol, tr->x[2], e2);
                res->edep += e2;
                continue;
            }
            track_t* c2 = &res->sec[res->n_sec++];
            c2->type = st;
            c2->T = sT;
            memcpy(c2->x, tr->x, sizeof tr->x);
            memcpy(c2->u, pr.dir[k], sizeof tr->u);
            c2->vol = tr->vol;
            c2->uid = orc_child_uid(h->seed, event_id, tr->uid, tr->step, (uint32_t)k);
            c2->step = 0;
        }
        if (!pr.null_interaction) {
            if (!pr.parent_alive) {
                alive = 0;
            } else if (tr->T < h->cut[tr->type]) {
                double e2 = tr->T + rest_energy(tr->type);
                deposit(h, ta, tr->vol, tr->x[2], e2);
                res->edep += e2;
                alive = 0;
            }
        }
    }
    /* 10 */
    tr->step += 1;
    if (alive && (int)tr->step >= h->max_steps) {
        ta->killed += tr->T + rest_energy(tr->type);
        alive = 0;
    }
    res->alive = alive;
}

typedef struct {
    track_t* v;
    size_t n, cap;
} stack_t_;

static void push(stack_t_* s, const track_t* t)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 1024;
        s->v = (track_t*)realloc(s->v, s->cap * sizeof(track_t));
    }
    s->v[s->n++] = *t;
}

/* transport one event depth-first from a stack (order does not change
 * any result: every track draws from its own counter-based stream) */
static void run_event(const orc_handle* h, uint64_t event_id, int n, const int* idx, const int32_t* type,
                      const double* T, const double* pos, const double* dir, tally_t* ta, uint64_t* step_hist,
                      int step_bins)
{
    stack_t_ st = {NULL, 0, 0};
    for (int i = n - 1; i >= 0; --i) {
        int p = idx[i];
        track_t t;
        t.type = type[p];
        t.T = T[p];
        for (int a = 0; a < 3; ++a) {
            t.x[a] = pos[3 * p + a];
            t.u[a] = dir[3 * p + a];
        }
        t.uid = (uint64_t)i + 1;
        t.step = 0;
        t.vol = locate(h, t.x);
        ta->e_in += t.T + rest_energy(t.type);
        if (t.vol == VOL_OUT) {
            ta->escaped += t.T + rest_energy(t.type);
            continue;
        }
        if (t.T < h->cut[t.type]) {
            deposit(h, ta, t.vol, t.x[2], t.T + rest_energy(t.type));
            continue;
        }
        push(&st, &t);
    }
    while (st.n > 0) {
        track_t t = st.v[--st.n];
        ta->n_tracks += 1.0;
        for (;;) {
            step_result_t r;
            step_track(h, event_id, &t, ta, &r);
            ta->n_steps += 1.0;
            for (int k = r.n_sec - 1; k >= 0; --k) push(&st, &r.sec[k]);
            if (!r.alive) break;
        }
        /* steps per track by particle type (Sec. 3.2 diagnostics) */
        if (step_hist) {
            uint32_t b = t.step < (uint32_t)(step_bins - 1) ? t.step : (uint32_t)(step_bins - 1);
            step_hist[(size_t)t.type * step_bins + b] += 1;
        }
    }
    free(st.v);
}

int orc_nav_exit(const orc_handle* h, int vol, const double* p, const double* d, double* t)
{
    exit_t e = nav_exit(h, vol, p, d);
    *t = e.t;
    return e.next;
}

int orc_locate(const orc_handle* h, const double* p) { return locate(h, p); }

int orc_step_one(orc_handle* h, double* trk, uint64_t uid, uint64_t event_id, double* sec, uint64_t* sec_uid,
                 double* info)
{
    track_t t;
    t.type = (int)trk[0];
    t.T = trk[1];
    for (int a = 0; a < 3; ++a) {
        t.x[a] = trk[2 + a];
        t.u[a] = trk[5 + a];
    }
    t.vol = (int)trk[8];
    t.step = (uint32_t)trk[9];
    t.uid = uid;
    double hist[4096];
    memset(hist, 0, sizeof hist);
    tally_t ta;
    memset(&ta, 0, sizeof ta);
    ta.hist = hist;
    step_result_t r;
    step_track(h, event_id, &t, &ta, &r);
    trk[0] = t.type;
    trk[1] = t.T;
    for (int a = 0; a < 3; ++a) {
        trk[2 + a] = t.x[a];
        trk[5 + a] = t.u[a];
    }
    trk[8] = t.vol;
    trk[9] = t.step;
    for (int k = 0; k < r.n_sec; ++k) {
        double* o = sec + 8 * k;
        o[0] = r.sec[k].type;
        o[1] = r.sec[k].T;
        for (int a = 0; a < 3; ++a) {
            o[2 + a] = r.sec[k].x[a];
            o[5 + a] = r.sec[k].u[a];
        }
        sec_uid[k] = r.sec[k].uid;
    }
    info[0] = r.s;
    info[1] = r.edep;
    info[2] = r.boundary;
    info[3] = r.interacted;
    info[4] = r.process;
    info[5] = r.alive;
    info[6] = ta.escaped;
    info[7] = ta.killed;
    return r.n_sec;
}

/* ---- thread pool over events ---- */
typedef struct {
    const orc_handle* h;
    int n_events;
    const uint64_t* event_ids;
    const int* start; /* CSR over primaries grouped by event */
    const int* order;
    const int32_t* type;
    const double *T, *pos, *dir;
    double* hist;
    double* summary;
    uint64_t* step_hist; /* [3][step_bins] or NULL */
    int step_bins;
    volatile int next;
    pthread_mutex_t mu;
} job_t;

static void* worker(void* arg)
{
    job_t* j = (job_t*)arg;
    uint64_t* sh = j->step_hist ? (uint64_t*)calloc((size_t)3 * j->step_bins, sizeof(uint64_t)) : NULL;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int e = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (e >= j->n_events) break;
        tally_t ta;
        memset(&ta, 0, sizeof ta);
        ta.hist = j->hist + (size_t)e * j->h->n_bins;
        memset(ta.hist, 0, sizeof(double) * j->h->n_bins);
        int b = j->start[e], n = j->start[e + 1] - b;
        run_event(j->h, j->event_ids[e], n, j->order + b, j->type, j->T, j->pos, j->dir, &ta, sh, j->step_bins);
        double* s = j->summary + 6 * (size_t)e;
        s[0] = ta.edep;
        s[1] = ta.escaped;
        s[2] = ta.killed;
        s[3] = ta.e_in;
        s[4] = ta.n_steps;
        s[5] = ta.n_tracks;
    }
    if (sh) {
        pthread_mutex_lock(&j->mu);
        for (int k = 0; k < 3 * j->step_bins; ++k) j->step_hist[k] += sh[k];
        pthread_mutex_unlock(&j->mu);
        free(sh);
    }
    return NULL;
}

int orc_run(orc_handle* h, int n_prim, const int32_t* ev, const int32_t* type, const double* T,
            const double* pos, const double* dir, int n_events, const uint64_t* event_ids, double* hist,
            double* summary, int n_threads, uint64_t* step_hist, int step_bins)
{
    if (step_hist && step_bins < 1) return -1;
    if (n_events <= 0) return 0;
    int* start = (int*)calloc((size_t)n_events + 1, sizeof(int));
    int* order = (int*)malloc(sizeof(int) * (size_t)(n_prim > 0 ? n_prim : 1));
    for (int i = 0; i < n_prim; ++i) {
        if (ev[i] < 0 || ev[i] >= n_events) {
            free(start);
            free(order);
            return -1;
        }
        start[ev[i] + 1]++;
    }
    for (int e = 0; e < n_events; ++e) start[e + 1] += start[e];
    int* fill = (int*)calloc((size_t)n_events, sizeof(int));
    for (int i = 0; i < n_prim; ++i) order[start[ev[i]] + fill[ev[i]]++] = i; /* submit order */
    free(fill);
    job_t j;
    j.h = h;
    j.n_events = n_events;
    j.event_ids = event_ids;
    j.start = start;
    j.order = order;
    j.type = type;
    j.T = T;
    j.pos = pos;
    j.dir = dir;
    j.hist = hist;
    j.summary = summary;
    j.step_hist = step_hist;
    j.step_bins = step_bins;
    j.next = 0;
    pthread_mutex_init(&j.mu, NULL);
    if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &j);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
    free(start);
    free(order);
    return 0;
}
