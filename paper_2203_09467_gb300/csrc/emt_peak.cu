// emt_peak.cu -- measured FP64 fused multiply-add throughput of the GPU, the
// denominator of the step kernels' arithmetic roofline (the FP64 step is
// led by the FP64 pipe, whose rate on GB300 is a small fraction of FP32's),
// and the throughput of FP64 division and logarithm, native and on the
// integer pipe.
//
// Every thread runs kChains independent chains x <- x * m + a (one DFMA
// each), so that the pipe, not the latency of one chain, sets the rate; the
// grid holds several full-occupancy waves of every SM.  The sums are stored
// so that no chain can be removed.  Measurement support only: the paper has
// no counterpart.
#include <cuda_runtime.h>

#include "../../include/emt.h"
#include "emt_intdiv.cuh"
#include "emt_intlog.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma_peak(double m, double a, int iters, double* out)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, a);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Throughput of FP64 division and logarithm, native and on the integer pipe
// (the step kernels' emt_intdiv.cuh and emt_intlog.cuh): kChains
// independent chains per thread.  Division: q = x / y, then x <- y,
// y <- q + 1.5 (operands stay in [1.5, 3.5]); logarithm: s += ln u for
// uniforms u from a 64-bit integer LCG.  Each operation carries one FP64
// addition.  kind: 0 native division, 1 integer division, 2 native log,
// 3 integer log.
template <int kind>
__global__ void __launch_bounds__(kThreads) k_op_rate(int iters, double* out)
{
    double x[kChains], y[kChains];
    unsigned long long st[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        x[k] = 1.5 + (double)((threadIdx.x * 7 + k * 3) & 15) * 0.0625;
        y[k] = 2.0 + (double)((threadIdx.x * 5 + k) & 15) * 0.0625;
        st[k] = 0x9E3779B97F4A7C15ull * (blockIdx.x * blockDim.x + threadIdx.x + 1) + k;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (kind < 2) {
                const double q = kind == 0 ? x[k] / y[k] : emt::intdiv::div_rn(x[k], y[k]);
                x[k] = y[k];
                y[k] = q + 1.5;
            } else {
                st[k] = st[k] * 6364136223846793005ull + 1442695040888963407ull;
                const double u = (double)((st[k] >> 11) | 1ull) * 0x1p-53;  // exact: an odd integer below 2^53
                x[k] += kind == 2 ? log(u) : emt::intlog::log_rn(u);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k] + y[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" emt_status emt_measure_fp64_op_rates(int32_t device, int32_t iters, int32_t repeats, double* rates)
{
    if (!rates || iters < 1 || repeats < 1) return EMT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return EMT_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        return EMT_ERR_CUDA;
    const int blocks = sms * 8;
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    emt_status rc = EMT_ERR_CUDA;
    if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        bool ok = true;
        for (int kind = 0; ok && kind < 4; ++kind) {
            auto launch = [&]() {
                if (kind == 0) k_op_rate<0><<<blocks, kThreads, 0, st>>>(iters, out);
                if (kind == 1) k_op_rate<1><<<blocks, kThreads, 0, st>>>(iters, out);
                if (kind == 2) k_op_rate<2><<<blocks, kThreads, 0, st>>>(iters, out);
                if (kind == 3) k_op_rate<3><<<blocks, kThreads, 0, st>>>(iters, out);
            };
            launch();  // warm-up
            double best = 0.0;
            ok = cudaGetLastError() == cudaSuccess;
            for (int r = 0; ok && r < repeats; ++r) {
                float ms = 0.f;
                ok = cudaEventRecord(e0, st) == cudaSuccess;
                launch();
                ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
                     cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                if (ok && ms > 0.f) {
                    const double rate = (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3);
                    if (rate > best) best = rate;
                }
            }
            rates[kind] = best;
            ok = ok && best > 0.0;
        }
        if (ok) rc = EMT_OK;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}

extern "C" emt_status emt_measure_dfma_rate(int32_t device, int32_t iters, int32_t repeats, double* fma_per_s)
{
    if (!fma_per_s || iters < 1 || repeats < 1) return EMT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return EMT_ERR_CUDA;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_peak, kThreads, 0) != cudaSuccess || sms < 1 ||
        per_sm < 1)
        return EMT_ERR_CUDA;
    const int blocks = sms * per_sm * 4;  // four full waves
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    emt_status rc = EMT_ERR_CUDA;
    if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kThreads) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        k_dfma_peak<<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, iters, out);  // warm-up
        double best = 0.0;
        bool ok = cudaGetLastError() == cudaSuccess;
        for (int r = 0; ok && r < repeats; ++r) {
            float ms = 0.f;
            ok = cudaEventRecord(e0, st) == cudaSuccess;
            k_dfma_peak<<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, iters, out);
            ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
                 cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && ms > 0.f) {
                const double rate = (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3);
                if (rate > best) best = rate;
            }
        }
        if (ok && best > 0.0) {
            *fma_per_s = best;
            rc = EMT_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}
