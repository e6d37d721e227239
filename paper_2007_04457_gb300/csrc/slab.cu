// Launchers of the slab load-vector kernel (slab.cuh), for FP32 level arrays
// with FP32 (plain) or FP64 (mixed precision) coarse arrays.
#include "launch.cuh"
#include "slab.cuh"

namespace mg {

namespace {

using SlabFn = void (*)(SlabParams);

// rows of up to 513 nodes: 256-thread blocks with registers for `minb`
// blocks per SM (3, or 2 with more registers); longer rows: 512 threads
template <typename TW, int TY, bool XS>
SlabFn slab_fn_xs(int n2, int minb)
{
    if ((n2 - 1) / 2 > 256) return k_slab<TW, TY, 512, 1, XS>;
    return minb >= 3 ? k_slab<TW, TY, 256, 3, XS> : k_slab<TW, TY, 256, 2, XS>;
}

template <typename TW, int TY>
SlabFn slab_fn_ty(int n2, int minb, bool xs)
{
    return xs ? slab_fn_xs<TW, TY, true>(n2, minb) : slab_fn_xs<TW, TY, false>(n2, minb);
}

template <typename TW>
SlabFn slab_fn(int ty, int n2, int minb, bool xs)
{
    switch (ty) {
    case 4: return slab_fn_ty<TW, 4>(n2, minb, xs);
    case 6: return slab_fn_ty<TW, 6>(n2, minb, xs);
    case 8: return slab_fn_ty<TW, 8>(n2, minb, xs);
    default: return nullptr;
    }
}

}  // namespace

int slab_slot_bytes_of(int ty, int n2)
{
    if (ty == 4) return slab_slot_bytes<4>(n2);
    if (ty == 6) return slab_slot_bytes<6>(n2);
    if (ty == 8) return slab_slot_bytes<8>(n2);
    return 0;
}

size_t slab_smem_bytes(int ty, int n2, int ns, bool xs, int tw_bytes)
{
    size_t b = (size_t)kSlabBarBytes + (size_t)ns * (size_t)slab_slot_bytes_of(ty, n2);
    if (xs)
        b += (size_t)(ty == 4 ? slab_xs_bytes<4>(n2, tw_bytes) : ty == 6 ? slab_xs_bytes<6>(n2, tw_bytes)
                                                                        : slab_xs_bytes<8>(n2, tw_bytes));
    return b;
}

template <typename TW>
cudaError_t slab_occupancy(int ty, int n2, int ns, int minb, bool xs, int *blocks_per_sm)
{
    auto fn = slab_fn<TW>(ty, n2, minb, xs);
    if (!fn || ns < 2 || ns > kSlabMaxSlots || (n2 - 1) % 64 != 0 || (n2 - 1) / 2 > kSlabMaxThreads)
        return cudaErrorInvalidValue;
    const size_t smem = slab_smem_bytes(ty, n2, ns, xs, (int)sizeof(TW));
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, (n2 - 1) / 2, smem);
}

template <typename TW>
cudaError_t launch_slab(int ty, int minb, bool xs, const SlabParams &p, int grid, cudaStream_t st)
{
    auto fn = slab_fn<TW>(ty, p.n2, minb, xs);
    if (!fn || p.nitems <= 0 || grid <= 0 || p.slot_bytes != slab_slot_bytes_of(ty, p.n2) || (xs && !p.fx))
        return cudaErrorInvalidValue;
    const size_t smem = slab_smem_bytes(ty, p.n2, p.ns, xs, (int)sizeof(TW));
    // the limit is per function: plans with other shapes may have lowered it
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return launch_pdl(fn, dim3(grid), dim3((p.n2 - 1) / 2), smem, st, p);
}

template cudaError_t slab_occupancy<float>(int, int, int, int, bool, int *);
template cudaError_t slab_occupancy<double>(int, int, int, int, bool, int *);
template cudaError_t launch_slab<float>(int, int, bool, const SlabParams &, int, cudaStream_t);
template cudaError_t launch_slab<double>(int, int, bool, const SlabParams &, int, cudaStream_t);

}  // namespace mg
