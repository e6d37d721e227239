// interp.cuh -- one-thread-per-node level kernels on an (x-chunk, row, plane)
// grid.
//
// k_scatter: after a decomposition level's coefficients are in place
//   (sweep.cuh), the N_{l-1} nodes receive the final coarse values V (Fig. 3:
//   each node keeps the value of the coarsest level it belongs to).
// node_iter serves the one-thread-per-node kernels of adjoint.cuh.
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

// One warp per row of N_{l-1} nodes (even row of an even plane): the row is
// read whole and written back whole with V in its even columns, so every
// written sector is complete (no partial-sector merges in L2).  Per chunk of
// 128 columns all loads are issued before the stores.
constexpr int kScatterWarps = 8;

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(32 * kScatterWarps) k_scatter(PlaceParams p)
{
    pdl_wait();
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const int L = threadIdx.x & 31;
    const int64_t rows = p.m0 * p.m1;
    const int64_t n2 = p.n2;
    for (int64_t row = (int64_t)blockIdx.x * kScatterWarps + (threadIdx.x >> 5); row < rows;
         row += (int64_t)gridDim.x * kScatterWarps) {
        const int64_t Z = row / p.m1, Y = row - (row / p.m1) * p.m1;
        const int64_t z = HZ ? 2 * Z : 0, y = HY ? 2 * Y : 0;
        T *arow = A + (z * p.n1 + y) * n2;
        const TW *vrow = V + row * p.m2;
        for (int64_t x0 = 0; x0 < n2; x0 += 128) {
            T a[4];
            TW v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t x = x0 + 32 * k + L;
                const bool in = x < n2;
                a[k] = (in && (x & 1)) ? arow[x] : T(0);
                v[k] = (in && !(x & 1)) ? vrow[x >> 1] : TW(0);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t x = x0 + 32 * k + L;
                if (x < n2) arow[x] = (x & 1) ? a[k] : static_cast<T>(v[k]);
            }
        }
    }
}

}  // namespace mg
