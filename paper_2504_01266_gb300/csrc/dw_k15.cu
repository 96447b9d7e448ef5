// Depthwise kernels instantiated for K = 15 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(15)
GIGA_DW_INSTANTIATE_BWD(15)
}  // namespace giga
