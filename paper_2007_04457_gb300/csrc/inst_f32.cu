// Kernel instantiations for FP32 storage and arithmetic.
#include "launch_impl.cuh"

namespace mg {
MG_INSTANTIATE_LEVEL(float, float)
MG_INSTANTIATE_SOLVE(float)
}  // namespace mg
