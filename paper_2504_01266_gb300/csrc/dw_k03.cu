// Depthwise kernels instantiated for K = 3 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(3)
GIGA_DW_INSTANTIATE_BWD(3)
}  // namespace giga
