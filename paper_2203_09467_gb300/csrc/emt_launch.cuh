// emt_launch.cuh -- host launchers of the step-loop kernels, instantiated
// once per precision in its own translation unit (different FMA flags).
#pragma once

#include "emt_internal.h"
#include "emt_step.cuh"

namespace emt {

template <typename R>
cudaError_t Launch<R>::step(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int block,
                            cudaStream_t st)
{
    if (block == 128)
        k_step<R, 128><<<grid, 128, 0, st>>>(p, side, cin, cout, cclr);
    else if (block == 256)
        k_step<R, 256><<<grid, 256, 0, st>>>(p, side, cin, cout, cclr);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::admit(const Params<R>& p, int side, int cs, int n, const int32_t* ev, const int32_t* type,
                             const double* T, const double* pos, const double* dir, const uint32_t* slot_of_event,
                             const uint32_t* uid_of, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_admit<R><<<(n + 255) / 256, 256, 0, st>>>(p, side, cs, n, ev, type, T, pos, dir, slot_of_event, uid_of);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::set_tracks(const Params<R>& p, int side, int cs, int n, const double* rec,
                                  const uint64_t* uid, const int32_t* slot, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_set_tracks<R><<<(n + 255) / 256, 256, 0, st>>>(p, side, cs, n, rec, uid, slot);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::get_tracks(const Params<R>& p, int side, int nG, int nC, double* rec, uint64_t* uid,
                                  int32_t* slot, cudaStream_t st)
{
    int n = nG + nC;
    if (n <= 0) return cudaSuccess;
    k_get_tracks<R><<<(n + 255) / 256, 256, 0, st>>>(p, side, nG, nC, rec, uid, slot);
    return cudaGetLastError();
}

template <typename R>
int Launch<R>::max_blocks_per_sm(int block)
{
    int n = 0;
    cudaError_t e = block == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<R, 128>, 128, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<R, 256>, 256, 0);
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace emt

#include "emt_split.cuh"

namespace emt {

template <typename R>
cudaError_t Launch<R>::step_split(const Params<R>& p, int side, int cin, int cout, int cclr, int grid_a, int grid_b,
                                  int block, cudaStream_t st)
{
    if (block == 128) {
        k_transport<R, 128><<<grid_a, 128, 0, st>>>(p, side, cin, cout, cclr);
        k_interact<R, 128><<<grid_b, 128, 0, st>>>(p, side, cin, cout);
    } else if (block == 256) {
        k_transport<R, 256><<<grid_a, 256, 0, st>>>(p, side, cin, cout, cclr);
        k_interact<R, 256><<<grid_b, 256, 0, st>>>(p, side, cin, cout);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R>
int Launch<R>::max_blocks_split(int block, int which)
{
    int n = 0;
    cudaError_t e;
    if (which == 0)
        e = block == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_transport<R, 128>, 128, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_transport<R, 256>, 256, 0);
    else
        e = block == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interact<R, 128>, 128, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_interact<R, 256>, 256, 0);
    if (e != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace emt
