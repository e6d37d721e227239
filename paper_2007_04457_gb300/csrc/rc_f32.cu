// Row-chunk kernel instantiations for FP32 storage and arithmetic.
#include "rc_launch.cuh"

namespace mg {
MG_INSTANTIATE_RC(float, float)
}  // namespace mg
