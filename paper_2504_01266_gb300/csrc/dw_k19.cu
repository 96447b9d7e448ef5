// Depthwise kernels instantiated for K = 19 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(19)

}  // namespace giga
