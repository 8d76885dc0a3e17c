// emt_launch.cuh -- host launchers of the step-loop kernels, instantiated
// once per precision in its own translation unit (different FMA flags).
#pragma once

#include "emt_internal.h"
#include "emt_step.cuh"

namespace emt {

// the physics options (multiple scattering, angular distributions,
// Rayleigh) select their own kernel instantiations
template <typename R>
static bool extended(const Params<R>& p)
{
    return (p.mask & (kProcMsc | kProcAngular | kProcRayleigh)) != 0u;
}

template <typename R, int BS, int G>
static void launch_fused(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, cudaStream_t st)
{
    if (extended(p))
        k_step<R, BS, G, true><<<grid, BS, 0, st>>>(p, side, cin, cout, cclr);
    else
        k_step<R, BS, G, false><<<grid, BS, 0, st>>>(p, side, cin, cout, cclr);
}

template <typename R>
cudaError_t Launch<R>::step(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int block,
                            cudaStream_t st)
{
    const bool cyl = p.geom == kGeomCylinders;
    if (block == 128) {
        if (cyl)
            launch_fused<R, 128, kGeomCylinders>(p, side, cin, cout, cclr, grid, st);
        else
            launch_fused<R, 128, kGeomLayers>(p, side, cin, cout, cclr, grid, st);
    } else if (block == 256) {
        if (cyl)
            launch_fused<R, 256, kGeomCylinders>(p, side, cin, cout, cclr, grid, st);
        else
            launch_fused<R, 256, kGeomLayers>(p, side, cin, cout, cclr, grid, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R, int BS, int G, bool X>
static cudaError_t launch_persist_x(const Params<R>& p, long long it0, int max_steps, GridSync* gs,
                                   long long limit_cycles, int grid, cudaStream_t st)
{
    Params<R> pc = p;
    void* args[] = {&pc, &it0, &max_steps, &gs, &limit_cycles};
    return cudaLaunchCooperativeKernel((const void*)k_persist<R, BS, G, X>, dim3(grid), dim3(BS), args, 0, st);
}

template <typename R>
cudaError_t Launch<R>::persist(const Params<R>& p, long long it0, int max_steps, GridSync* gs,
                               long long limit_cycles, int grid, int block, cudaStream_t st)
{
    const bool cyl = p.geom == kGeomCylinders;
    const bool x = extended(p);
    if (block == 128) {
        if (cyl)
            return x ? launch_persist_x<R, 128, kGeomCylinders, true>(p, it0, max_steps, gs, limit_cycles, grid, st)
                     : launch_persist_x<R, 128, kGeomCylinders, false>(p, it0, max_steps, gs, limit_cycles, grid, st);
        return x ? launch_persist_x<R, 128, kGeomLayers, true>(p, it0, max_steps, gs, limit_cycles, grid, st)
                 : launch_persist_x<R, 128, kGeomLayers, false>(p, it0, max_steps, gs, limit_cycles, grid, st);
    }
    if (block == 256) {
        if (cyl)
            return x ? launch_persist_x<R, 256, kGeomCylinders, true>(p, it0, max_steps, gs, limit_cycles, grid, st)
                     : launch_persist_x<R, 256, kGeomCylinders, false>(p, it0, max_steps, gs, limit_cycles, grid, st);
        return x ? launch_persist_x<R, 256, kGeomLayers, true>(p, it0, max_steps, gs, limit_cycles, grid, st)
                 : launch_persist_x<R, 256, kGeomLayers, false>(p, it0, max_steps, gs, limit_cycles, grid, st);
    }
    return cudaErrorInvalidValue;
}

// resident blocks per SM of the persistent kernel, the smallest over its
// instantiations (every block of a cooperative launch must be resident)
template <typename R, int BS>
static int min_blocks_persist()
{
    int n[4] = {0, 0, 0, 0};
    cudaError_t e[4];
    e[0] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], k_persist<R, BS, kGeomLayers, false>, BS, 0);
    e[1] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], k_persist<R, BS, kGeomCylinders, false>, BS, 0);
    e[2] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[2], k_persist<R, BS, kGeomLayers, true>, BS, 0);
    e[3] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[3], k_persist<R, BS, kGeomCylinders, true>, BS, 0);
    int m = 1 << 30;
    for (int k = 0; k < 4; ++k) {
        if (e[k] != cudaSuccess) return 0;
        if (n[k] < m) m = n[k];
    }
    return m;
}

template <typename R>
int Launch<R>::persist_blocks_per_sm(int block)
{
    return block == 128 ? min_blocks_persist<R, 128>() : min_blocks_persist<R, 256>();
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
cudaError_t Launch<R>::unspill(const Params<R>& p, int side, int cs, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_unspill<R><<<(n + 255) / 256, 256, 0, st>>>(p, side, cs, n);
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

// resident blocks per SM of the fused kernel, the smallest over its
// instantiations (geometry kind x physics options)
template <typename R, int BS>
static int min_blocks_fused()
{
    int n[4] = {0, 0, 0, 0};
    cudaError_t e[4];
    e[0] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], k_step<R, BS, kGeomLayers, false>, BS, 0);
    e[1] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], k_step<R, BS, kGeomCylinders, false>, BS, 0);
    e[2] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[2], k_step<R, BS, kGeomLayers, true>, BS, 0);
    e[3] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[3], k_step<R, BS, kGeomCylinders, true>, BS, 0);
    int m = 1 << 30;
    for (int k = 0; k < 4; ++k) {
        if (e[k] != cudaSuccess) return 1;
        if (n[k] < m) m = n[k];
    }
    return m > 0 ? m : 1;
}

template <typename R>
int Launch<R>::max_blocks_per_sm(int block)
{
    return block == 128 ? min_blocks_fused<R, 128>() : min_blocks_fused<R, 256>();
}

}  // namespace emt

#include "emt_split.cuh"

namespace emt {

template <typename R, int BS, bool S, bool X>
static void launch_split_x(const Params<R>& p, int side, int cin, int cout, int cclr, int grid_a, int grid_b,
                           cudaStream_t st)
{
    if (!S && p.has_field) {
        // charged tracks sorted by expected substep count (k_transport takes
        // them in that order)
        k_sort_keys<R><<<grid_b, 256, 0, st>>>(p, side, cin);
        k_sort_order<R><<<grid_b, 256, 0, st>>>(p, cin);
    }
    if (p.geom == kGeomCylinders)
        k_transport<R, BS, kGeomCylinders, S, X><<<grid_a, BS, 0, st>>>(p, side, cin, cout, cclr);
    else
        k_transport<R, BS, kGeomLayers, S, X><<<grid_a, BS, 0, st>>>(p, side, cin, cout, cclr);
    k_interact<R, BS, S, X><<<grid_b, BS, 0, st>>>(p, side, cin, cout);
}

template <typename R, int BS, bool S>
static void launch_split(const Params<R>& p, int side, int cin, int cout, int cclr, int grid_a, int grid_b,
                         cudaStream_t st)
{
    if (extended(p))
        launch_split_x<R, BS, S, true>(p, side, cin, cout, cclr, grid_a, grid_b, st);
    else
        launch_split_x<R, BS, S, false>(p, side, cin, cout, cclr, grid_a, grid_b, st);
}

template <typename R>
cudaError_t Launch<R>::step_split(const Params<R>& p, int side, int cin, int cout, int cclr, int grid_a, int grid_b,
                                  int block, cudaStream_t st)
{
    const bool sel = p.max_active > 0;
    if (block == 128) {
        if (sel)
            launch_split<R, 128, true>(p, side, cin, cout, cclr, grid_a, grid_b, st);
        else
            launch_split<R, 128, false>(p, side, cin, cout, cclr, grid_a, grid_b, st);
    } else if (block == 256) {
        if (sel)
            launch_split<R, 256, true>(p, side, cin, cout, cclr, grid_a, grid_b, st);
        else
            launch_split<R, 256, false>(p, side, cin, cout, cclr, grid_a, grid_b, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// resident blocks per SM of the split kernels (which 0: transport, 1:
// interaction), the smallest over the instantiations
template <typename R, int BS>
static int min_blocks_split(int which)
{
    int n[8];
    cudaError_t e[8];
    int k = 0;
    if (which == 0) {
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomLayers, false, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomCylinders, false, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomLayers, true, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomCylinders, true, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomLayers, false, true>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomCylinders, false, true>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomLayers, true, true>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_transport<R, BS, kGeomCylinders, true, true>, BS, 0), ++k;
    } else {
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_interact<R, BS, false, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_interact<R, BS, true, false>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_interact<R, BS, false, true>, BS, 0), ++k;
        e[k] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[k], k_interact<R, BS, true, true>, BS, 0), ++k;
    }
    int m = 1 << 30;
    for (int j = 0; j < k; ++j) {
        if (e[j] != cudaSuccess) return 1;
        if (n[j] < m) m = n[j];
    }
    return m > 0 ? m : 1;
}

template <typename R>
int Launch<R>::max_blocks_split(int block, int which)
{
    return block == 128 ? min_blocks_split<R, 128>(which) : min_blocks_split<R, 256>(which);
}

template <typename R, int BS, bool X>
static void launch_pipe_x(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int grid_sort,
                          cudaStream_t st)
{
    if (p.has_field) {
        k_sort_keys<R><<<grid_sort, 256, 0, st>>>(p, side, cin);
        k_sort_order<R><<<grid_sort, 256, 0, st>>>(p, cin);
    }
    if (p.geom == kGeomCylinders)
        k_pipe<R, BS, kGeomCylinders, X><<<grid, BS, 0, st>>>(p, side, cin, cout, cclr);
    else
        k_pipe<R, BS, kGeomLayers, X><<<grid, BS, 0, st>>>(p, side, cin, cout, cclr);
}

template <typename R>
cudaError_t Launch<R>::step_pipe(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int grid_sort,
                                 int block, cudaStream_t st)
{
    const bool x = extended(p);
    if (block == 128) {
        if (x)
            launch_pipe_x<R, 128, true>(p, side, cin, cout, cclr, grid, grid_sort, st);
        else
            launch_pipe_x<R, 128, false>(p, side, cin, cout, cclr, grid, grid_sort, st);
    } else if (block == 256) {
        if (x)
            launch_pipe_x<R, 256, true>(p, side, cin, cout, cclr, grid, grid_sort, st);
        else
            launch_pipe_x<R, 256, false>(p, side, cin, cout, cclr, grid, grid_sort, st);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// resident blocks per SM of the pipelined kernel, the smallest over its
// instantiations
template <typename R, int BS>
static int min_blocks_pipe()
{
    int n[4] = {0, 0, 0, 0};
    cudaError_t e[4];
    e[0] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[0], k_pipe<R, BS, kGeomLayers, false>, BS, 0);
    e[1] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[1], k_pipe<R, BS, kGeomCylinders, false>, BS, 0);
    e[2] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[2], k_pipe<R, BS, kGeomLayers, true>, BS, 0);
    e[3] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n[3], k_pipe<R, BS, kGeomCylinders, true>, BS, 0);
    int m = 1 << 30;
    for (int k = 0; k < 4; ++k) {
        if (e[k] != cudaSuccess) return 1;
        if (n[k] < m) m = n[k];
    }
    return m > 0 ? m : 1;
}

template <typename R>
int Launch<R>::max_blocks_pipe(int block)
{
    return block == 128 ? min_blocks_pipe<R, 128>() : min_blocks_pipe<R, 256>();
}

}  // namespace emt

// Explicit instantiations, split across translation units so that the
// heavy kernel families compile in parallel.
#define EMT_INSTANTIATE_FUSED(R)                                                                                    \
    template cudaError_t Launch<R>::step(const Params<R>&, int, int, int, int, int, int, cudaStream_t);           \
    template cudaError_t Launch<R>::admit(const Params<R>&, int, int, int, const int32_t*, const int32_t*,         \
                                          const double*, const double*, const double*, const uint32_t*,         \
                                          const uint32_t*, cudaStream_t);                                         \
    template cudaError_t Launch<R>::set_tracks(const Params<R>&, int, int, int, const double*, const uint64_t*,   \
                                               const int32_t*, cudaStream_t);                                     \
    template cudaError_t Launch<R>::get_tracks(const Params<R>&, int, int, int, double*, uint64_t*, int32_t*,     \
                                               cudaStream_t);                                                     \
    template int Launch<R>::max_blocks_per_sm(int);                                                               \
    template cudaError_t Launch<R>::unspill(const Params<R>&, int, int, int, cudaStream_t);
#define EMT_INSTANTIATE_PERSIST(R)                                                                                  \
    template cudaError_t Launch<R>::persist(const Params<R>&, long long, int, GridSync*, long long, int, int,     \
                                            cudaStream_t);                                                        \
    template int Launch<R>::persist_blocks_per_sm(int);
#define EMT_INSTANTIATE_SPLIT(R)                                                                                    \
    template cudaError_t Launch<R>::step_split(const Params<R>&, int, int, int, int, int, int, int, cudaStream_t); \
    template int Launch<R>::max_blocks_split(int, int);
#define EMT_INSTANTIATE_PIPE(R)                                                                                     \
    template cudaError_t Launch<R>::step_pipe(const Params<R>&, int, int, int, int, int, int, int, cudaStream_t);  \
    template int Launch<R>::max_blocks_pipe(int);
