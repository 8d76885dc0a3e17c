// emt_tables.cu -- builds every cross-section, stopping-power and range
// table on the device, in FP64 (compiled with --fmad=false).
//
// Tables are tabulated on the log grid E_n = E_lo 10^(n/bpd) (Sec. 2.2: all
// particle types use tabulated cross sections).  The paper prints no model
// formula; these are the textbook closed forms:
//   radiation length   Tsai 1974 (PDG review "Passage of particles through
//                      matter", Eq. 34.26)
//   Compton            Klein-Nishina total cross section
//   pair production    Bethe-Heitler, complete screening (PDG Eq. 34.31),
//                      integrated over x in [me/k, 1 - me/k]
//   photoelectric      Sauter high-energy K-shell limit x 5/4
//   bremsstrahlung     Tsai complete screening (PDG Eq. 34.29 without y^2/9)
//   ionisation         Moller (e-) and Bhabha (e+) integrated above the cut
//   annihilation       Heitler two-photon in flight
//   stopping power     Berger-Seltzer restricted collision loss (ICRU 37)
//                      with the high-energy density-effect asymptote, plus
//                      the radiative loss below the photon cut
//   range              R_0 = E_0/S(E_0); R_n = R_{n-1} + int dE/S by
//                      16-point Gauss-Legendre in ln E on each interval,
//                      split at the energies where S has a kink.
#include <cuda_runtime.h>

#include "emt_device.cuh"
#include "emt_internal.h"

namespace emt {

namespace {

__device__ double x0_gcm2(double Z, double A)
{
    double a = kAlpha * Z;
    double a2 = a * a;
    double fz = a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
    double z13 = cbrt(Z);
    double lrad = log(184.15 / z13);
    double lprad = log(1194.0 / (z13 * z13));
    double inv = 4.0 * kAlpha * kRe * kRe * (kNa / A) * (Z * Z * (lrad - fz) + Z * lprad);
    return 1.0 / inv;
}

__device__ double sigma_kn(double k)
{
    double kappa = k / kMe;
    double a = 1.0 + 2.0 * kappa;
    double l = log(a);
    double t1 = (1.0 + kappa) / (kappa * kappa) * (2.0 * (1.0 + kappa) / a - l / kappa);
    double t2 = l / (2.0 * kappa);
    double t3 = (1.0 + 3.0 * kappa) / (a * a);
    return 2.0 * kPi * kRe * kRe * (t1 + t2 - t3);
}

__device__ double sigma_photo_atom(double Z, double k, double bk)
{
    if (k <= bk) return 0.0;
    double a2 = kAlpha * kAlpha;
    double z5 = Z * Z * Z * Z * Z;
    return 5.0 * kPi * kRe * kRe * (a2 * a2) * z5 * (kMe / k);
}

__device__ double sigma_moller(double T, double cut)
{
    if (T <= 2.0 * cut) return 0.0;
    double xc = cut / T;
    double g = (T + kMe) / kMe;
    double b2 = T * (T + 2.0 * kMe) / ((T + kMe) * (T + kMe));
    double g1 = (g - 1.0) / g;
    double c = (2.0 * g - 1.0) / (g * g);
    double br = g1 * g1 * (0.5 - xc) + 1.0 / xc - 1.0 / (1.0 - xc) - c * log((1.0 - xc) / xc);
    return 2.0 * kPi * kRe * kRe * kMe / (b2 * T) * br;
}

__device__ double sigma_bhabha(double T, double cut)
{
    if (T <= cut) return 0.0;
    double xc = cut / T;
    double g = (T + kMe) / kMe;
    double y = 1.0 / (g + 1.0);
    double y2 = y * y;
    double t = 1.0 - 2.0 * y;
    double b2 = T * (T + 2.0 * kMe) / ((T + kMe) * (T + kMe));
    double c1 = 2.0 - y2;
    double c2 = t * (3.0 + y2);
    double c4 = t * t * t;
    double c3 = t * t + c4;
    double br = (1.0 / xc - 1.0) / b2 + c1 * log(xc) + c2 * (1.0 - xc) - c3 * (1.0 - xc * xc) / 2.0 +
                c4 * (1.0 - xc * xc * xc) / 3.0;
    return 2.0 * kPi * kRe * kRe * kMe / T * br;
}

// Rayleigh scattering: Thomson scattering off the atom with the form factor
// of an exponentially screened charge, F = Z / (1 + (q a)^2)^2, screening
// radius a = 0.88534 a0 Z^(-1/3).  With x = 1 - cos, b = 2 (k a / hbar c)^2,
// sigma = pi re^2 Z^2 I(b), I(b) = int_0^2 (2 - 2x + x^2) (1 + b x)^-4 dx:
// its Taylor series below b = 0.1 (the closed form cancels there), else
// [A (1 - Y^-3)/3 + B (1 - Y^-2)/2 + C (1 - Y^-1)] / b with Y = 1 + 2b,
// A = 2 + 2/b + 1/b^2, B = -2/b - 2/b^2, C = 1/b^2 (substituting y = 1 + b x).
__device__ double rayleigh_screening(double Z) { return 0.88534 * kBohr / cbrt(Z); }

__device__ double sigma_rayleigh_atom(double Z, double k)
{
    const double y = k * rayleigh_screening(Z) / kHbarC;
    const double b = 2.0 * y * y;
    double I;
    if (b < 0.1) {
        double sum = 0.0, bn = 1.0, p2 = 4.0;  // p2 = 2^(n+2)
        for (int n = 0; n < 40; ++n) {
            const double mn = p2 / (n + 1.0) - 2.0 * p2 / (n + 2.0) + 2.0 * p2 / (n + 3.0);
            const double c = (n + 1.0) * (n + 2.0) * (n + 3.0) / 6.0;
            sum += ((n & 1) ? -c : c) * bn * mn;
            bn *= b;
            p2 *= 2.0;
        }
        I = sum;
    } else {
        const double Y = 1.0 + 2.0 * b;
        const double A = 2.0 + 2.0 / b + 1.0 / (b * b), B = -2.0 / b - 2.0 / (b * b), C = 1.0 / (b * b);
        const double y1 = 1.0 / Y, y2 = y1 * y1, y3 = y2 * y1;
        I = (A * (1.0 - y3) / 3.0 + B * (1.0 - y2) / 2.0 + C * (1.0 - y1)) / b;
    }
    return kPi * kRe * kRe * Z * Z * I;
}

__device__ double sigma_heitler(double T)
{
    double tau = T / kMe;
    double g = tau + 1.0;
    double gg1 = tau * (tau + 2.0);
    double s = sqrt(gg1);
    return kPi * kRe * kRe / (g + 1.0) * ((g * g + 4.0 * g + 1.0) / gg1 * log(g + s) - (g + 3.0) / s);
}

__device__ double sigma_brems_macro(double x0_cm, double T, double kc)
{
    if (T <= kc) return 0.0;
    double E = T + kMe;
    return 1.0 / x0_cm * (4.0 / 3.0 * log(T / kc) - 4.0 / 3.0 * (T - kc) / E + (T * T - kc * kc) / (2.0 * E * E));
}

__device__ double dedx_rad(double x0_cm, double T, double kc)
{
    double E = T + kMe;
    double kp = kc < T ? kc : T;
    return 1.0 / x0_cm * (4.0 / 3.0 * kp - 2.0 / 3.0 * kp * kp / E + kp * kp * kp / (3.0 * E * E));
}

__device__ double dedx_coll(const MaterialDev& m, int charge, double T, double cut)
{
    double nel = m.rho * kNa / m.A * m.Z;
    double tau = T / kMe;
    double g = tau + 1.0;
    double b2 = tau * (tau + 2.0) / (g * g);
    double Im = m.I_eV * 1e-6 / kMe;
    double F;
    if (charge < 0) {
        double dmax = 0.5 * T;
        double D = (cut < dmax ? cut : dmax) / kMe;
        F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D) +
            (0.5 * D * D + (2.0 * tau + 1.0) * log(1.0 - D / tau)) / (g * g);
    } else {
        double D = (cut < T ? cut : T) / kMe;
        double y = 1.0 / (tau + 2.0);
        double D2 = D * D, D3 = D2 * D, D4 = D3 * D;
        double y2 = y * y, y3 = y2 * y;
        F = log(tau * D) -
            b2 / tau * (tau + 2.0 * D - 1.5 * D2 * y - (D - D3 / 3.0) * y2 - (0.5 * D2 - tau * D3 / 3.0 + 0.25 * D4) * y3);
    }
    double hwp = 28.816 * sqrt(m.rho * m.Z / m.A);
    double bg = sqrt(tau * (tau + 2.0));
    double delta = 2.0 * log(bg) + 2.0 * log(hwp / m.I_eV) - 1.0;
    if (delta < 0.0) delta = 0.0;
    double S = 2.0 * kPi * kRe * kRe * kMe * nel / b2 * (log(2.0 * (tau + 2.0) / (Im * Im)) + F - delta);
    if (S < 1e-12) S = 1e-12;
    return S;
}

__device__ double dedx_total(const MaterialDev& m, double x0_cm, int p, double T, double cut_e, double kc)
{
    double coll = dedx_coll(m, p == 1 ? -1 : 1, T, cut_e);
    return coll + dedx_rad(x0_cm, T, kc);
}

// Gauss-Legendre nodes (ascending) and weights by Newton's method on P_16
// from the Chebyshev-like guess cos(pi (i + 3/4)/(n + 1/2))
__global__ void k_gauss_legendre(double* x, double* w)
{
    const int n = 16;
    int i = threadIdx.x;
    if (i >= n) return;
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

__global__ void k_grid(TableBuild b)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= b.n_grid) return;
    b.grid[n] = b.e_lo * pow(10.0, (double)n / b.bpd);
}

// one thread per (material, node): cross sections and stopping powers
__global__ void k_xs(TableBuild b)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= b.n_mat * b.n_grid) return;
    int mi = idx / b.n_grid, n = idx % b.n_grid;
    const MaterialDev m = b.mats[mi];
    double* t0 = b.tab + ((size_t)(mi * 3 + 0) * b.n_grid + n) * kNq;
    double* t1 = b.tab + ((size_t)(mi * 3 + 1) * b.n_grid + n) * kNq;
    double* t2 = b.tab + ((size_t)(mi * 3 + 2) * b.n_grid + n) * kNq;
    for (int q = 0; q < kNq; ++q) {
        t0[q] = 0.0;
        t1[q] = 0.0;
        t2[q] = 0.0;
    }
    b.dedx[(size_t)(mi * 3 + 0) * b.n_grid + n] = 0.0;
    b.dedx[(size_t)(mi * 3 + 1) * b.n_grid + n] = 0.0;
    b.dedx[(size_t)(mi * 3 + 2) * b.n_grid + n] = 0.0;
    if (!(m.rho > 0.0)) return;
    const double n_at = m.rho * kNa / m.A;
    const double n_el = m.Z * n_at;
    const double x0_cm = x0_gcm2(m.Z, m.A) / m.rho;
    const double E = b.grid[n];
    const double kc = b.cut[0], cut_e = b.cut[1];
    const unsigned mask = b.mask;
    if (mask & 1u) t0[0] = n_at * sigma_photo_atom(m.Z, E, m.bk);
    if (mask & 2u) t0[1] = n_el * sigma_kn(E);
    if (mask & 4u) {
        double s = 0.0;
        if (E > 2.0 * kMe) {
            double hh = 0.5 - kMe / E;
            s = (4.0 / 3.0 * hh + 8.0 / 9.0 * hh * hh * hh) / x0_cm;
        }
        t0[2] = s;
    }
    if (mask & kProcRayleigh) t0[3] = n_at * sigma_rayleigh_atom(m.Z, E);
    if (mask & 8u) t1[0] = n_el * sigma_moller(E, cut_e);
    if (mask & 16u) t1[1] = sigma_brems_macro(x0_cm, E, kc);
    b.dedx[(size_t)(mi * 3 + 1) * b.n_grid + n] = dedx_total(m, x0_cm, 1, E, cut_e, kc);
    if (mask & 8u) t2[0] = n_el * sigma_bhabha(E, cut_e);
    if (mask & 16u) t2[1] = sigma_brems_macro(x0_cm, E, kc);
    if (mask & 32u) t2[2] = n_el * sigma_heitler(E);
    b.dedx[(size_t)(mi * 3 + 2) * b.n_grid + n] = dedx_total(m, x0_cm, 2, E, cut_e, kc);
}

// one thread per (material, charged particle, interval i >= 1): int dE/S
__global__ void k_range_intervals(TableBuild b, const double* glx, const double* glw, double* acc)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int per = b.n_grid;
    if (idx >= b.n_mat * 2 * per) return;
    int i = idx % per;
    int pm = idx / per;
    int mi = pm / 2, p = 1 + pm % 2;
    acc[idx] = 0.0;
    const MaterialDev m = b.mats[mi];
    if (i == 0 || !(m.rho > 0.0)) return;
    const double x0_cm = x0_gcm2(m.Z, m.A) / m.rho;
    const double kc = b.cut[0], cut_e = b.cut[1];
    double hwp = 28.816 * sqrt(m.rho * m.Z / m.A);
    double bg0 = exp(0.5) * m.I_eV / hwp;
    double t_dens = kMe * (sqrt(1.0 + bg0 * bg0) - 1.0);
    double k3[3] = {p == 1 ? 2.0 * cut_e : cut_e, kc, t_dens};
    for (int x = 0; x < 3; ++x)
        for (int y = x + 1; y < 3; ++y)
            if (k3[y] < k3[x]) {
                double t = k3[x];
                k3[x] = k3[y];
                k3[y] = t;
            }
    double edges[5];
    int ne = 0;
    edges[ne++] = b.grid[i - 1];
    for (int x = 0; x < 3; ++x)
        if (k3[x] > edges[ne - 1] && k3[x] < b.grid[i]) edges[ne++] = k3[x];
    edges[ne++] = b.grid[i];
    double a_acc = 0.0;
    for (int sub = 0; sub + 1 < ne; ++sub) {
        double a = log(edges[sub]), bb = log(edges[sub + 1]);
        double half = 0.5 * (bb - a), mid = 0.5 * (a + bb);
        double sum = 0.0;
        for (int j = 0; j < 16; ++j) {
            double E = exp(mid + half * glx[j]);
            sum += glw[j] * (E / dedx_total(m, x0_cm, p, E, cut_e, kc));
        }
        a_acc += half * sum;
    }
    acc[idx] = a_acc;
}

// one thread per (material, charged particle): ordered prefix sum into R
__global__ void k_range_scan(TableBuild b, const double* acc)
{
    int pm = blockIdx.x * blockDim.x + threadIdx.x;
    if (pm >= b.n_mat * 2) return;
    int mi = pm / 2, p = 1 + pm % 2;
    if (!(b.mats[mi].rho > 0.0)) return;
    double* t = b.tab + (size_t)(mi * 3 + p) * b.n_grid * kNq;
    const double* S = b.dedx + (size_t)(mi * 3 + p) * b.n_grid;
    const double* a = acc + (size_t)pm * b.n_grid;
    double R = b.grid[0] / S[0];
    t[3] = R;
    for (int i = 1; i < b.n_grid; ++i) {
        R = R + a[i];
        t[i * kNq + 3] = R;
    }
}

__global__ void k_to_float(const double* src, float* dst, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

// differences of consecutive nodes, v[(row * n + i) * q + j]: d = v[i+1] - v[i]
// (0 at the last node); the interpolations use them as b - a, the same
// value the subtraction gives at lookup time
template <typename T>
__global__ void k_node_diff(const T* v, T* d, int total, int n, int q)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (idx / q) % n;
    d[idx] = i + 1 < n ? v[idx + q] - v[idx] : T(0);
}

}  // namespace

// reciprocal interval widths of the energy grid and of the range tables
// (interpolation fractions are products with them, as in the oracle)
__global__ void k_reciprocals(TableBuild b)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = b.n_grid;
    if (idx < n) b.igrid[idx] = idx + 1 < n ? 1.0 / (b.grid[idx + 1] - b.grid[idx]) : 0.0;
    if (idx >= b.n_mat * 3 * n) return;
    const int row = idx / n, i = idx % n;
    const int p = row % 3;
    double v = 0.0;
    if (p > 0 && i + 1 < n && b.mats[row / 3].rho > 0.0) {
        const double* t = b.tab + (size_t)row * n * kNq;
        v = 1.0 / (t[(i + 1) * kNq + 3] - t[i * kNq + 3]);
    }
    b.irs[idx] = v;
}

__global__ void k_x0(TableBuild b)
{
    const int i = threadIdx.x;
    if (i >= b.n_mat) return;
    const MaterialDev& m = b.mats[i];
    b.x0[i] = m.rho > 0.0 ? x0_gcm2(m.Z, m.A) / m.rho : 0.0;
    if (b.ray_a) b.ray_a[i] = m.rho > 0.0 ? rayleigh_screening(m.Z) : 0.0;
}

cudaError_t build_tables(const TableBuild& b, double* scratch, cudaStream_t st)
{
    if (b.x0) k_x0<<<1, 32, 0, st>>>(b);
    // scratch: 32 doubles of Gauss-Legendre data + n_mat*2*n_grid interval integrals
    double* glx = scratch;
    double* glw = scratch + 16;
    double* acc = scratch + 32;
    k_gauss_legendre<<<1, 32, 0, st>>>(glx, glw);
    k_grid<<<(b.n_grid + 127) / 128, 128, 0, st>>>(b);
    int nx = b.n_mat * b.n_grid;
    k_xs<<<(nx + 127) / 128, 128, 0, st>>>(b);
    int ni = b.n_mat * 2 * b.n_grid;
    k_range_intervals<<<(ni + 127) / 128, 128, 0, st>>>(b, glx, glw, acc);
    k_range_scan<<<1, 64, 0, st>>>(b, acc);
    const int nr = b.n_mat * 3 * b.n_grid;
    k_reciprocals<<<(nr + 127) / 128, 128, 0, st>>>(b);
    const int nt = b.n_mat * 3 * b.n_grid * kNq;
    k_node_diff<<<(nt + 255) / 256, 256, 0, st>>>(b.tab, b.dtab, nt, b.n_grid, kNq);
    k_node_diff<<<(b.n_grid + 255) / 256, 256, 0, st>>>(b.grid, b.dgrid, b.n_grid, b.n_grid, 1);
    if (b.tabf) {
        k_to_float<<<(nt + 255) / 256, 256, 0, st>>>(b.tab, b.tabf, nt);
        k_to_float<<<(b.n_grid + 255) / 256, 256, 0, st>>>(b.grid, b.gridf, b.n_grid);
        k_to_float<<<(b.n_grid + 255) / 256, 256, 0, st>>>(b.igrid, b.igridf, b.n_grid);
        k_to_float<<<(nr + 255) / 256, 256, 0, st>>>(b.irs, b.irsf, nr);
        k_node_diff<<<(nt + 255) / 256, 256, 0, st>>>(b.tabf, b.dtabf, nt, b.n_grid, kNq);
        k_node_diff<<<(b.n_grid + 255) / 256, 256, 0, st>>>(b.gridf, b.dgridf, b.n_grid, b.n_grid, 1);
    }
    return cudaGetLastError();
}

}  // namespace emt
