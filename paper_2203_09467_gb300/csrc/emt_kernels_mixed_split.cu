// emt_kernels_mixed_split.cu -- mixed-precision instantiation of the split schedule's transport and interaction kernels.
// Built with FMA contraction enabled.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_SPLIT(float)
}
