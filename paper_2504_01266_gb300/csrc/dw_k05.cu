// Depthwise kernels instantiated for K = 5 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(5)
GIGA_DW_INSTANTIATE_BWD(5)
}  // namespace giga
