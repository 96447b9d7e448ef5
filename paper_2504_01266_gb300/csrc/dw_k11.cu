// Depthwise kernels instantiated for K = 11 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(11)
GIGA_DW_INSTANTIATE_BWD(11)
}  // namespace giga
