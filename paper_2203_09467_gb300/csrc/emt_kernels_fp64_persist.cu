// emt_kernels_fp64_persist.cu -- FP64 instantiation of the persistent step loop.
// Built with --fmad=false (see emt_kernels_fp64.cu).
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_PERSIST(double)
}
