// Persistent batch kernel instantiations: user arrays of type float, arithmetic in float.
#include "persist_launch.cuh"

namespace mg {
MG_INSTANTIATE_PERSIST(float, float)
}  // namespace mg
