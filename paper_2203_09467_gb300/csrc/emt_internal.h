// emt_internal.h -- declarations shared by the library's translation units
// (host runtime, table builder, FP64 and mixed-precision step kernels).
#pragma once

#include <cuda_runtime.h>

#include "emt_device.cuh"

namespace emt {

struct MaterialDev {
    double Z, A, rho, I_eV, bk;
};

struct TableBuild {
    double* x0;               // [n_mat] radiation length (cm), 0 for vacuum (optional)
    double* ray_a;            // [n_mat] Rayleigh screening radius (cm) (optional)
    const MaterialDev* mats;  // device
    int n_mat;
    int n_grid;
    int bpd;
    double e_lo;
    double cut[3];
    unsigned mask;
    double* grid;  // [n_grid]
    double* tab;   // [n_mat][3][n_grid][4]
    double* dedx;  // [n_mat][3][n_grid]
    float* tabf;   // optional float copies (mixed precision)
    float* gridf;
    double* igrid;  // [n_grid] 1 / (grid[n+1] - grid[n]) (last entry 0)
    double* irs;    // [n_mat][3][n_grid] 1 / (R[n+1] - R[n]) of the range tables
    float* igridf;  // optional float copies
    float* irsf;
    double* dgrid;  // [n_grid] grid[n+1] - grid[n] (last entry 0)
    double* dtab;   // [n_mat][3][n_grid][4] tab[n+1][q] - tab[n][q] (last node 0)
    float* dgridf;  // optional: the same differences of the float copies, in float
    float* dtabf;
};

// scratch: (32 + n_mat * 2 * n_grid) doubles
cudaError_t build_tables(const TableBuild& b, double* scratch, cudaStream_t st);

template <typename R>
struct Launch {
    static cudaError_t step(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int block,
                            cudaStream_t st);
    static cudaError_t admit(const Params<R>& p, int side, int cs, int n, const int32_t* ev, const int32_t* type,
                             const double* T, const double* pos, const double* dir, const uint32_t* slot_of_event,
                             const uint32_t* uid_of, cudaStream_t st);
    static cudaError_t set_tracks(const Params<R>& p, int side, int cs, int n, const double* rec,
                                  const uint64_t* uid, const int32_t* slot, cudaStream_t st);
    static cudaError_t get_tracks(const Params<R>& p, int side, int nG, int nC, double* rec, uint64_t* uid,
                                  int32_t* slot, cudaStream_t st);
    static int max_blocks_per_sm(int block);
    // split schedule: transport kernel then interaction kernel
    static cudaError_t step_split(const Params<R>& p, int side, int cin, int cout, int cclr, int grid_a, int grid_b,
                                  int block, cudaStream_t st);
    static int max_blocks_split(int block, int which);
    // pipelined schedule: one kernel per step (plus the two sorting launches
    // of the charged tracks in a field, on grid_sort blocks)
    static cudaError_t step_pipe(const Params<R>& p, int side, int cin, int cout, int cclr, int grid, int grid_sort,
                                 int block, cudaStream_t st);
    static int max_blocks_pipe(int block);
    // host spill: append n tracks of the spill buffer to side `side`
    static cudaError_t unspill(const Params<R>& p, int side, int cs, int n, cudaStream_t st);
    // persistent step loop (fused schedule, cooperative launch of `grid`
    // resident blocks): up to max_steps steps from global iteration it0
    static cudaError_t persist(const Params<R>& p, long long it0, int max_steps, GridSync* gs,
                               long long limit_cycles, int grid, int block, cudaStream_t st);
    static int persist_blocks_per_sm(int block);
};

// diagnostics: a bounded grid wait that is never released (on `blocks`
// blocks); sets kStatusTimeout in *status once it gives up
cudaError_t launch_wait_never(GridSync* gs, long long limit_cycles, int* status, int blocks, cudaStream_t st);

}  // namespace emt
