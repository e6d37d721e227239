// rc_launch.cuh -- launchers of the row-chunk level kernels (rowchunk.cuh),
// included only by the rc_*.cu translation units (one per element-type
// combination, compiled in parallel).
#pragma once

#include <algorithm>

#include "launch.cuh"
#include "rowchunk.cuh"

namespace mg {

namespace rcdetail {

using Fn = void (*)(RcParams);

template <typename T, typename TW, int Q>
Fn sweep_fn(int mode, bool hz, bool wu)
{
    if (mode == MODE_DEC) {
        if (hz) return wu ? k_rc_sweep<T, TW, Q, true, MODE_DEC, true> : k_rc_sweep<T, TW, Q, true, MODE_DEC, false>;
        return wu ? k_rc_sweep<T, TW, Q, false, MODE_DEC, true> : k_rc_sweep<T, TW, Q, false, MODE_DEC, false>;
    }
    if (hz) return wu ? k_rc_sweep<T, TW, Q, true, MODE_REC, true> : k_rc_sweep<T, TW, Q, true, MODE_REC, false>;
    return wu ? k_rc_sweep<T, TW, Q, false, MODE_REC, true> : k_rc_sweep<T, TW, Q, false, MODE_REC, false>;
}

template <typename T, typename TW, int Q, bool HZ>
Fn restrict_fn_hz(bool ku, bool xs)
{
    constexpr int TY = kRcRows;
    if (ku) return xs ? k_rc_restrict<T, TW, Q, HZ, true, true, TY> : k_rc_restrict<T, TW, Q, HZ, true, false, TY>;
    return xs ? k_rc_restrict<T, TW, Q, HZ, false, true, TY> : k_rc_restrict<T, TW, Q, HZ, false, false, TY>;
}

template <typename T, typename TW, int Q>
Fn restrict_fn(bool hz, bool ku, bool xs)
{
    return hz ? restrict_fn_hz<T, TW, Q, true>(ku, xs) : restrict_fn_hz<T, TW, Q, false>(ku, xs);
}

template <typename T, typename TW, int Q>
Fn pick_q(int kind, int mode, bool hz, bool u, bool xs)
{
    return kind == 0 ? sweep_fn<T, TW, Q>(mode, hz, u) : restrict_fn<T, TW, Q>(hz, u, xs);
}

// sub-segments per segment compiled per element type: segments of 256 and
// 512 columns for 4-byte elements (Q = 2, 4), 256 for 8-byte ones (Q = 4)
template <typename T, typename TW>
Fn pick(int kind, int Q, int mode, bool hz, bool u, bool xs)
{
    if constexpr (sizeof(T) == 4) {
        if (Q == 2) return pick_q<T, TW, 2>(kind, mode, hz, u, xs);
        if (Q == 4) return pick_q<T, TW, 4>(kind, mode, hz, u, xs);
    } else {
        if (Q == 4) return pick_q<T, TW, 4>(kind, mode, hz, u, xs);
    }
    return nullptr;
}

template <typename T, typename TW, int Q>
size_t smem_q(int kind, int mode, int S, bool u, bool xs)
{
    if (kind == 0) return mode == MODE_DEC ? rc_sweep_smem<T, TW, Q, MODE_DEC>() : rc_sweep_smem<T, TW, Q, MODE_REC>();
    return rc_restrict_smem<T, TW, Q>(S, u, xs);
}

template <typename T, typename TW>
size_t smem_of(int kind, int Q, int mode, int S, bool u, bool xs)
{
    if constexpr (sizeof(T) == 4) {
        if (Q == 2) return smem_q<T, TW, 2>(kind, mode, S, u, xs);
        return smem_q<T, TW, 4>(kind, mode, S, u, xs);
    } else {
        return smem_q<T, TW, 4>(kind, mode, S, u, xs);
    }
}

}  // namespace rcdetail

template <typename T, typename TW>
cudaError_t rc_occupancy(int kind, int Q, int mode, bool hz, bool u, bool xs, int S, int *blocks_per_sm)
{
    rcdetail::Fn fn = rcdetail::pick<T, TW>(kind, Q, mode, hz, u, xs);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = rcdetail::smem_of<T, TW>(kind, Q, mode, S, u, xs);
    if (smem > 0) {
        cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 32 * kRcWarps, smem);
}

template <typename T, typename TW>
cudaError_t launch_rc(int kind, int Q, int mode, bool hz, bool u, bool xs, const RcParams &p, int grid,
                      cudaStream_t st)
{
    rcdetail::Fn fn = rcdetail::pick<T, TW>(kind, Q, mode, hz, u, xs);
    if (!fn || p.nitems <= 0 || grid <= 0) return cudaErrorInvalidValue;
    const size_t smem = rcdetail::smem_of<T, TW>(kind, Q, mode, p.S, u, xs);
    if (smem > 0) {
        // the limit is per function: plans with other shapes may have lowered it
        cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    return launch_pdl(fn, dim3(grid), dim3(32 * kRcWarps), smem, st, p);
}

#define MG_INSTANTIATE_RC(T, TW)                                                                            \
    template cudaError_t rc_occupancy<T, TW>(int, int, int, bool, bool, bool, int, int *);                  \
    template cudaError_t launch_rc<T, TW>(int, int, int, bool, bool, bool, const RcParams &, int, cudaStream_t);

}  // namespace mg
