// Persistent batch kernel instantiations: user arrays of type float, arithmetic in double.
#include "persist_launch.cuh"

namespace mg {
MG_INSTANTIATE_PERSIST(float, double)
}  // namespace mg
