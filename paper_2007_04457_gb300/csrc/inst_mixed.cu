// Kernel instantiations for the finest level of the mixed-precision scheme:
// FP32 field and stencil arithmetic, FP64 coarse arrays and load vector.
#include "launch_impl.cuh"

namespace mg {
MG_INSTANTIATE_LEVEL(float, double)
}  // namespace mg
