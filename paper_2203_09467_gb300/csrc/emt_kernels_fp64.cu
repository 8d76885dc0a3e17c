// emt_kernels_fp64.cu -- FP64 instantiation of the fused step kernel and
// the small kernels (the other families: emt_kernels_fp64_{persist,split,
// pipe}.cu).  Built with --fmad=false: every FP64 expression rounds exactly
// as written, so the path reproduces the FP64 CPU oracle operation by
// operation.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_FUSED(double)

// Diagnostics: a barrier that is never reached (it waits for one block
// more than the launch has), so that every block's bounded wait runs out
// and sets kStatusTimeout; the kernel then ends normally.
__global__ void k_wait_never(GridSync* gs, long long limit_cycles, int* status)
{
    grid_barrier(gs, gridDim.x + 1u, limit_cycles, status);
}

cudaError_t launch_wait_never(GridSync* gs, long long limit_cycles, int* status, int blocks, cudaStream_t st)
{
    k_wait_never<<<blocks, 32, 0, st>>>(gs, limit_cycles, status);
    return cudaGetLastError();
}
}  // namespace emt
