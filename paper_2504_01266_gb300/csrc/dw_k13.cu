// Depthwise kernels instantiated for K = 13 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(13)
GIGA_DW_INSTANTIATE_BWD(13)
}  // namespace giga
