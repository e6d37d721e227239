// Persistent batch kernel instantiations: user arrays of type double, arithmetic in double.
#include "persist_launch.cuh"

namespace mg {
MG_INSTANTIATE_PERSIST(double, double)
}  // namespace mg
