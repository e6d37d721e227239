// Row-chunk kernel instantiations for FP32 storage with FP64 coarse arrays.
#include "rc_launch.cuh"

namespace mg {
MG_INSTANTIATE_RC(float, double)
}  // namespace mg
