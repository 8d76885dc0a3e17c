// Test helper: Philox4x32-10 outputs of NVIDIA's cuRAND device API for
// given keys and counters (an independent implementation to check the
// oracle's generator against; run, not read).
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_philox(const uint32_t* key, const uint32_t* ctr, int n, uint32_t* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    unsigned long long seed = ((unsigned long long)key[2 * i + 1] << 32) | key[2 * i];
    unsigned long long subseq = ((unsigned long long)ctr[4 * i + 3] << 32) | ctr[4 * i + 2];
    unsigned long long off = ((unsigned long long)ctr[4 * i + 1] << 32) | ctr[4 * i + 0];
    curand_init(seed, subseq, 0, &st);
    skipahead((unsigned long long)4 * off, &st);
    uint4 v = curand4(&st);
    out[4 * i + 0] = v.x;
    out[4 * i + 1] = v.y;
    out[4 * i + 2] = v.z;
    out[4 * i + 3] = v.w;
}

extern "C" int curand_philox(const uint32_t* key, const uint32_t* ctr, int n, uint32_t* out)
{
    uint32_t *dk, *dc, *dout;
    if (cudaMalloc(&dk, 8 * n) || cudaMalloc(&dc, 16 * n) || cudaMalloc(&dout, 16 * n)) return 1;
    cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    k_philox<<<(n + 127) / 128, 128>>>(dk, dc, n, dout);
    cudaError_t e = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(dk);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 2;
}
