// GPU checks of the step kernels' integer-pipe FP64 arithmetic: the
// division (emt_intdiv.cuh) bit for bit against the native FP64 division on
// n pseudo-random operand pairs in the same regimes as the host check
// (tests/csrc/intdiv_host.cpp), and the logarithm (emt_intlog.cuh) against
// the native FP64 log, counting the arguments where the two differ and by
// how much.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../paper_2203_09467_gb300/csrc/emt_intdiv.cuh"
#include "../../paper_2203_09467_gb300/csrc/emt_intlog.cuh"

using emt::intdiv::bitsd;
using emt::intdiv::dbits;

__device__ __forceinline__ uint64_t mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_check(uint64_t n, uint64_t seed, unsigned long long* counts, double* ex)
{
    const uint64_t kM = (1ull << 52) - 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long nf = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t a = mix(seed ^ (3 * i)), b = mix(seed ^ (3 * i + 1)), c = mix(seed ^ (3 * i + 2));
        switch (i & 7) {
        case 1: b = (b & kM) | (1023ull << 52); break;
        case 2: b = (1023ull << 52) | (c & 0xF); break;
        case 3: b = (1023ull << 52) | (kM - (c & 0xF)); break;
        case 4: a = (a & ~kM) | (b & kM); break;
        case 5: a = (1023ull << 52) | (kM - (c & 0xFF)); break;
        case 6:
            a = (a & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(923 + c % 200) << 52);
            b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(923 + (c >> 32) % 200) << 52);
            break;
        case 7:
            b = (b & 0x800FFFFFFFFFFFFFull & ~0xFFFFFFFFull) | ((uint64_t)(1000 + c % 40) << 52);
            a = dbits(bitsd(b) * bitsd((1023ull << 52) | ((c >> 8) & kM & ~0xFFFFFFFFFull)));
            break;
        default: break;
        }
        const double x = bitsd(a), y = bitsd(b);
        const int e1 = (int)((a >> 52) & 0x7FF), e2 = (int)((b >> 52) & 0x7FF), er = e1 - e2 + 1023;
        if (!((unsigned)(e1 - 1) >= 2046u || (unsigned)(e2 - 1) >= 2046u || (unsigned)(er - 2) >= 2044u)) ++nf;
        const double q0 = x / y, q1 = emt::intdiv::div_rn(x, y);
        // and the square root of |x| (sign bit cleared), of y and of y^2
        const double ax = bitsd(a & 0x7FFFFFFFFFFFFFFFull), y2 = y * y;
        const bool sq_ok = dbits(sqrt(ax)) == dbits(emt::intdiv::sqrt_rn(ax)) &&
                           dbits(sqrt(fabs(y))) == dbits(emt::intdiv::sqrt_rn(fabs(y))) &&
                           (dbits(sqrt(y2)) == dbits(emt::intdiv::sqrt_rn(y2)) || y2 != y2);
        if (!sq_ok) atomicAdd(&counts[2], 1ull);
        if (dbits(q0) != dbits(q1) && !(q0 != q0 && q1 != q1)) {
            const unsigned long long k = atomicAdd(&counts[1], 1ull);
            if (k < 4) {
                ex[4 * k] = x;
                ex[4 * k + 1] = y;
                ex[4 * k + 2] = q0;
                ex[4 * k + 3] = q1;
            }
        }
    }
    atomicAdd(&counts[0], nf);
}

// counts[0] = operand pairs on the integer path, counts[1] = quotient
// mismatches, counts[2] = pairs with a square-root mismatch (of |x|, |y| or
// y^2); ex receives up to four quotient mismatches (x, y, native, integer);
// returns a CUDA error code
extern "C" int intdiv_check(unsigned long long n, unsigned long long seed, unsigned long long* counts, double* ex)
{
    unsigned long long* dc = nullptr;
    double* dex = nullptr;
    if (cudaMalloc(&dc, 3 * sizeof(unsigned long long)) != cudaSuccess) return 1;
    if (cudaMalloc(&dex, 16 * sizeof(double)) != cudaSuccess) return 1;
    cudaMemset(dc, 0, 3 * sizeof(unsigned long long));
    cudaMemset(dex, 0, 16 * sizeof(double));
    k_check<<<152 * 8, 256>>>(n, seed, dc, dex);
    cudaError_t e = cudaMemcpy(counts, dc, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ex, dex, 16 * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dex);
    return (int)e;
}

// counts[0] = arguments, counts[1] = results that differ from the native
// log, counts[2] = results more than one unit in the last place apart;
// ex receives up to four differing cases (x, native, integer)
__global__ void k_log_check(uint64_t n, uint64_t seed, unsigned long long* counts, double* ex)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long nd = 0, nb = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t w = mix(seed ^ i);
        double x;
        switch (i & 3) {
        case 0: x = (double)(2 * (w >> 12) + 1) * 0x1p-53; break;
        case 1: x = 1.0 - (double)((w >> 20) + 1) * 0x1p-53; break;
        case 2: x = 1.0 + (double)((w >> 20) + 1) * 0x1p-52; break;
        default: x = bitsd(((w >> 2) & 0x7FEFFFFFFFFFFFFFull) | 0x0010000000000000ull); break;
        }
        const double a = log(x), b = emt::intlog::log_rn(x);
        if (dbits(a) != dbits(b)) {
            ++nd;
            const long long d = (long long)(dbits(a) - dbits(b));
            if (d > 1 || d < -1) ++nb;
            const unsigned long long k = atomicAdd(&counts[3], 1ull);
            if (k < 4) {
                ex[3 * k] = x;
                ex[3 * k + 1] = a;
                ex[3 * k + 2] = b;
            }
        }
    }
    atomicAdd(&counts[1], nd);
    atomicAdd(&counts[2], nb);
}

extern "C" int intlog_check(unsigned long long n, unsigned long long seed, unsigned long long* counts, double* ex)
{
    unsigned long long* dc = nullptr;
    double* dex = nullptr;
    if (cudaMalloc(&dc, 4 * sizeof(unsigned long long)) != cudaSuccess) return 1;
    if (cudaMalloc(&dex, 12 * sizeof(double)) != cudaSuccess) return 1;
    cudaMemset(dc, 0, 4 * sizeof(unsigned long long));
    cudaMemset(dex, 0, 12 * sizeof(double));
    k_log_check<<<152 * 8, 256>>>(n, seed, dc, dex);
    cudaError_t e = cudaMemcpy(counts, dc, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ex, dex, 12 * sizeof(double), cudaMemcpyDeviceToHost);
    counts[0] = n;
    cudaFree(dc);
    cudaFree(dex);
    return (int)e;
}
