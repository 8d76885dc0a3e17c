// emt_peak.cu -- measured FP64 fused multiply-add throughput of the GPU, the
// denominator of the step kernels' arithmetic roofline (the FP64 step is
// led by the FP64 pipe, whose rate on GB300 is a small fraction of FP32's).
//
// Every thread runs kChains independent chains x <- x * m + a (one DFMA
// each), so that the pipe, not the latency of one chain, sets the rate; the
// grid holds several full-occupancy waves of every SM.  The sums are stored
// so that no chain can be removed.  Measurement support only: the paper has
// no counterpart.
#include <cuda_runtime.h>

#include "../../include/emt.h"

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

}  // namespace

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
