// emt_kernels_fp64_pipe.cu -- FP64 instantiation of the pipelined schedule's kernel.
// Built with --fmad=false (see emt_kernels_fp64.cu).
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_PIPE(double)
}
