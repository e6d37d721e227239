// persist_launch.cuh -- launcher of the persistent batch kernel (persist.cuh),
// included only by the persist_*.cu translation units (one per element-type
// combination, compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "params.h"
#include "persist.cuh"

namespace mg {

template <typename TX, typename TW>
cudaError_t persist_occupancy(int mode, size_t smem, int *blocks_per_sm)
{
    void (*fn)(PersistParams) = (mode == MODE_DEC) ? k_persist<TX, TW, MODE_DEC> : k_persist<TX, TW, MODE_REC>;
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kPersistThreads, smem);
}

template <typename TX, typename TW>
cudaError_t launch_persist(int mode, const PersistParams &p, int grid, size_t smem, cudaStream_t st)
{
    void (*fn)(PersistParams) = (mode == MODE_DEC) ? k_persist<TX, TW, MODE_DEC> : k_persist<TX, TW, MODE_REC>;
    if (grid <= 0) return cudaErrorInvalidValue;
    // the limit is per function: batches with other fields may have lowered it
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    fn<<<grid, kPersistThreads, smem, st>>>(p);
    return cudaGetLastError();
}

#define MG_INSTANTIATE_PERSIST(TX, TW)                                                       \
    template cudaError_t persist_occupancy<TX, TW>(int, size_t, int *);                      \
    template cudaError_t launch_persist<TX, TW>(int, const PersistParams &, int, size_t, cudaStream_t);

}  // namespace mg
