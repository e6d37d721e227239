// Row-chunk kernel instantiations for FP64 storage and arithmetic.
#include "rc_launch.cuh"

namespace mg {
MG_INSTANTIATE_RC(double, double)
}  // namespace mg
