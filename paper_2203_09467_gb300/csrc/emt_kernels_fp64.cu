// emt_kernels_fp64.cu -- FP64 instantiation of the step-loop kernels.
// Built with --fmad=false: every FP64 expression rounds exactly as written,
// so the path reproduces the FP64 CPU oracle operation by operation.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
template struct Launch<double>;
}
