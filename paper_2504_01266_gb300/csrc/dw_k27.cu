// Depthwise kernels instantiated for K = 27 (one translation unit per filter
// size so the build compiles them in parallel).
#include "dw_launch_impl.cuh"

namespace giga {
GIGA_DW_INSTANTIATE(27)

}  // namespace giga
