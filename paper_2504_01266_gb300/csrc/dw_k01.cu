// Depthwise kernels instantiated for K = 1 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(1)
GIGA_DW_INSTANTIATE_BWD(1)
}  // namespace giga
