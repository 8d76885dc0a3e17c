// emt_kernels_mixed_pipe.cu -- mixed-precision instantiation of the pipelined schedule's kernel.
// Built with FMA contraction enabled.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_PIPE(float)
}
