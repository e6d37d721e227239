// Kernel instantiations for FP64 storage and arithmetic (also the coarse
// levels of the mixed-precision scheme).
#include "launch_impl.cuh"

namespace mg {
MG_INSTANTIATE_LEVEL(double, double)
MG_INSTANTIATE_SOLVE(double)
}  // namespace mg
