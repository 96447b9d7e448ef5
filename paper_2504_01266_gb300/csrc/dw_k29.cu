// Depthwise kernels instantiated for K = 29 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(29)

}  // namespace giga
