// emt_kernels_mixed.cu -- mixed-precision instantiation of the fused step
// kernel and the small kernels (the other families: emt_kernels_mixed_
// {persist,split,pipe}.cu): FP32 tables, sampling and kinematics; FP64
// positions, boundary distances and energy tallies.  Built with FMA
// contraction enabled.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_FUSED(float)
}
