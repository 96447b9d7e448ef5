// Depthwise kernels instantiated for K = 7 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(7)
GIGA_DW_INSTANTIATE_BWD(7)
}  // namespace giga
