// emt_kernels_fp64_split.cu -- FP64 instantiation of the split schedule's transport and interaction kernels.
// Built with --fmad=false (see emt_kernels_fp64.cu).
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_SPLIT(double)
}
