// emt_kernels_mixed_persist.cu -- mixed-precision instantiation of the persistent step loop.
// Built with FMA contraction enabled.
#include "emt_internal.h"
#include "emt_launch.cuh"

namespace emt {
EMT_INSTANTIATE_PERSIST(float)
}
