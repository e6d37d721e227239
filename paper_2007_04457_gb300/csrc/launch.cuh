// launch.cuh -- host-side launchers of the level kernels, instantiated per
// element-type combination in inst_*.cu (compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "params.h"

namespace mg {

// Tile shapes of the fused restriction kernel selectable per level (coarse
// nodes in dims 1 x 2; a last tile absorbs the final node of a dimension):
//   2D/3D: cfg 0 = 8 x 64, cfg 1 = 4 x 64, cfg 2 = 16 x 64;  1D: 64
constexpr int kRestrictConfigs = 3;

struct RestrictShape {
    int ty, tx;          // coarse nodes per tile in dims 1 and 2
    size_t smem;         // dynamic shared memory bytes
    int blocks_per_sm;   // occupancy of the instantiation
};

template <typename T, typename TW>
cudaError_t restrict_shape(int act, int mode, int cfg, RestrictShape *out);

template <typename T, typename TW>
cudaError_t launch_restrict(int act, int mode, int cfg, const RestrictParams &p, int grid,
                            cudaStream_t st);

// Chunk length for a line of m nodes.  Lines of up to 288 nodes use register
// chunks of 16 (at most 18 warps per block); longer lines use 32
// shared-memory chunks of ceil(m/32).  Returns 0 when m exceeds kMaxLine.
constexpr int kMaxLine = 4096;
constexpr int kRegLine = 288;
inline int solve_chunk(int m)
{
    if (m <= kRegLine) return 16;
    if (m <= kMaxLine) return (m + 31) / 32;
    return 0;
}

// contiguous = lines along the fastest dimension (staged through shared
// memory when it fits, otherwise read directly).
template <typename TW>
cudaError_t launch_solve(const SolveParams &p, bool contiguous, bool use_smem, cudaStream_t st);

// phase 0: rows odd in dim 0 or 1; phase 1: even rows (see k_place)
template <typename T, typename TW>
cudaError_t launch_place(int act, int phase, const PlaceParams &p, int grid, cudaStream_t st);

template <typename T, typename TW>
cudaError_t launch_interp(int act, const PlaceParams &p, int grid, cudaStream_t st);

}  // namespace mg
