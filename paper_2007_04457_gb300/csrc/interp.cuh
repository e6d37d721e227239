// interp.cuh -- one-thread-per-node level kernels on an (x-chunk, row, plane)
// grid.
//
// k_scatter: after a decomposition level's coefficients are in place
//   (sweep.cuh), the N_{l-1} nodes receive the final coarse values V (Fig. 3:
//   each node keeps the value of the coarsest level it belongs to).
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kRowThreads = 256;

// Grid of the element-wise kernels: x in chunks of blockDim.x, dims 1 and 0
// in blockIdx.y / blockIdx.z with strided loops beyond 65535.
struct NodeIter {
    int64_t x, y0, z0, ystep, zstep;
};

__device__ __forceinline__ NodeIter node_iter()
{
    NodeIter it;
    it.x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    it.y0 = blockIdx.y;
    it.z0 = blockIdx.z;
    it.ystep = gridDim.y;
    it.zstep = gridDim.z;
    return it;
}

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kRowThreads) k_scatter(PlaceParams p)
{
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const NodeIter it = node_iter();
    const int64_t X = it.x;
    if (X >= p.m2) return;
    for (int64_t Z = it.z0; Z < p.m0; Z += it.zstep) {
        const int64_t z = HZ ? 2 * Z : 0;
        for (int64_t Y = it.y0; Y < p.m1; Y += it.ystep) {
            const int64_t y = HY ? 2 * Y : 0;
            A[(z * p.n1 + y) * p.n2 + 2 * X] = static_cast<T>(V[(Z * p.m1 + Y) * p.m2 + X]);
        }
    }
}

}  // namespace mg
