// emt_kernels_mixed.cu -- mixed-precision instantiation of the step-loop
// kernels: FP32 tables, sampling and kinematics; FP64 positions, boundary
// distances and energy tallies.  Built with FMA contraction enabled.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
template struct Launch<float>;
}
