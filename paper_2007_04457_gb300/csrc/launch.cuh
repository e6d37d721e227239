// launch.cuh -- host-side launchers of the level kernels, instantiated per
// element-type combination in inst_*.cu (compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "params.h"
#include "multi_params.h"
#include "persist_params.h"
#include "small_params.h"

namespace mg {

// Launch with programmatic dependent launch allowed: the kernel may start
// while its predecessor on the stream finishes, so it must call pdl_wait()
// (common.cuh) before it touches memory the predecessor writes or reads.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, args...);
}

// Tile shapes of the load-vector kernel selectable per level (coarse nodes in
// dims 1 x 2; a last tile absorbs the final node of a dimension):
//   2D/3D: cfg 0 = 8 x 64, cfg 1 = 4 x 64, cfg 2 = 16 x 64 (a block per tile),
//   cfg 3 = 8 x 30 (FP64: 4 x 30) per warp, for levels with m2 >= 30 and
//   m1 >= the strip rows;  1D: 256 per block
constexpr int kRestrictConfigs = 4;

struct RestrictShape {
    int ty, tx;            // coarse nodes per tile in dims 1 and 2
    size_t smem;           // dynamic shared memory bytes
    int blocks_per_sm;     // occupancy of the instantiation
    int items_per_block;   // work items a block runs at once
};

template <typename T, typename TW>
cudaError_t restrict_shape(int act, int mode, int cfg, RestrictShape *out);

template <typename T, typename TW>
cudaError_t launch_restrict(int act, int mode, int cfg, const RestrictParams &p, int grid,
                            cudaStream_t st);

// Longest coarse line the solve kernel takes (a panel of one line must fit in
// shared memory).
constexpr int kMaxLine = 4096;

// Solves along dimension k of a compact array; nw_req = 0: register-chunk
// kernel (16 or 32 nodes per warp) for lines up to 576 nodes; nw_req > 0:
// the shared-memory panel kernel with that many warps (chunks) per line.
template <typename TW>
cudaError_t launch_solve(const SolveParams &p, int nw_req, int num_sms, cudaStream_t st);

// Element-wise kernels: coefficients of a decomposed level (warp-tile
// sweep), placement of its final coarse values (one thread per coarse node),
// and recomposition of a level (warp-tile sweep).
template <typename T, typename TW>
cudaError_t launch_coef(int act, const PlaceParams &p, int num_sms, cudaStream_t st);

template <typename T, typename TW>
cudaError_t launch_scatter(int act, const PlaceParams &p, cudaStream_t st);

template <typename T, typename TW>
cudaError_t launch_interp(int act, const PlaceParams &p, int num_sms, cudaStream_t st);

// All remaining levels of a small array in one block (small.cuh); smem =
// small_elems(n) * sizeof(TW) bytes of dynamic shared memory.
template <typename T, typename TW>
cudaError_t launch_small(int mode, const SmallParams &p, size_t smem, cudaStream_t st);

// The coarse levels in one cooperative launch (multi.cuh): blocks of the
// kernel resident per SM with `smem` bytes of dynamic shared memory, and the
// launch itself (grid <= that count x the SM count).
template <typename TX, typename TW>
cudaError_t multi_occupancy(int mode, size_t smem, int *blocks_per_sm);

template <typename TX, typename TW>
cudaError_t launch_multi(int mode, const MultiParams &p, int grid, size_t smem, cudaStream_t st);

// Transposed maps of all remaining levels of a small array in one block
// (small.cuh): dir 0 = decomposition, 1 = recomposition; smem as launch_small.
template <typename T, typename TW>
cudaError_t launch_small_adj(int dir, const SmallParams &p, size_t smem, cudaStream_t st);

// Transposed level maps (adjoint.cuh).
template <typename T, typename TW>
cudaError_t launch_gather(int act, const PlaceParams &p, cudaStream_t st);

template <typename T, typename TW>
cudaError_t launch_adj_odd(int act, const AdjParams &p, cudaStream_t st);

template <typename T, typename TW>
cudaError_t launch_adj_even(int act, const AdjParams &p, cudaStream_t st);

// Finest-grid values of a level-k function from its compact values
// (prolong.cuh); p.shift >= 1, p.seg is set here.
template <typename T, typename TW>
cudaError_t launch_prolong(const ProlongParams &p, int num_sms, cudaStream_t st);


// Row-chunk level kernels (rowchunk.cuh): kind 0 = sweep (mode MODE_DEC:
// coefficients, MODE_REC: interpolation), kind 1 = load vector + coarse
// gather (xs: with the dim-2 solve).  Q = sub-segments of 32 words per
// segment (4-byte level arrays: 2 or 4, segments of 256 or 512 columns;
// 8-byte: 4, segments of 256), hz = 3D, u = uniform interpolation weights (sweep) or
// K_2 rows (restriction) along dim 2.
template <typename T, typename TW>
cudaError_t rc_occupancy(int kind, int Q, int mode, bool hz, bool u, bool xs, int S, int *blocks_per_sm);

template <typename T, typename TW>
cudaError_t launch_rc(int kind, int Q, int mode, bool hz, bool u, bool xs, const RcParams &p, int grid,
                      cudaStream_t st);

// The persistent batch kernel (persist.cuh): blocks resident per SM with
// `smem` bytes of dynamic shared memory, and the launch (any grid: its items
// never wait on an item no block holds).
template <typename TX, typename TW>
cudaError_t persist_occupancy(int mode, size_t smem, int *blocks_per_sm);

template <typename TX, typename TW>
cudaError_t launch_persist(int mode, const PersistParams &p, int grid, size_t smem, cudaStream_t st);

// Load vector + coarse gather of a 3D FP32 level from whole-row slabs staged
// by bulk asynchronous copies (slab.cuh): ty = coarse rows per band (4, 6
// or 8), ns = ring slots (2 .. kSlabMaxSlots), rows of n2 = 64 k + 1 nodes
// (k <= 16), blocks of (n2 - 1) / 2 threads; minb = 3 compiles rows of up
// to 513 nodes for three blocks per SM (fewer registers), else two.
constexpr int kSlabMaxSlots = 16;
constexpr int kSlabMaxThreads = 512;  // rows of up to 1025 nodes
int slab_slot_bytes_of(int ty, int n2);
size_t slab_smem_bytes(int ty, int n2, int ns, bool xs, int tw_bytes);

template <typename TW>
cudaError_t slab_occupancy(int ty, int n2, int ns, int minb, bool xs, int *blocks_per_sm);

// xs: the kernel also solves M_{l-1} along dim 2 (p.fx) before storing F
template <typename TW>
cudaError_t launch_slab(int ty, int minb, bool xs, const SlabParams &p, int grid, cudaStream_t st);

}  // namespace mg
