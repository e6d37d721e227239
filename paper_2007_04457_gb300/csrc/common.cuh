// common.cuh -- device helpers shared by the sm_103a kernels of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mg {

// Asynchronous global -> shared copy of one 4- or 8-byte element
// (cp.async, L1-allocating).  When `valid` is false no byte is read and the
// destination is zero-filled; `gmem` must still be a valid address.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem, bool valid)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int nbytes = valid ? static_cast<int>(sizeof(T)) : 0;
    if constexpr (sizeof(T) == 4) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes)
                     : "memory");
    } else {
        static_assert(sizeof(T) == 8, "4- or 8-byte elements");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes)
                     : "memory");
    }
}

// L2 policy that marks lines for early eviction (streamed data read once).
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}

// cp_async_elem with an L2 cache policy.
template <typename T>
__device__ __forceinline__ void cp_async_elem_hint(T *smem, const T *gmem, bool valid, uint64_t pol)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int nbytes = valid ? static_cast<int>(sizeof(T)) : 0;
    if constexpr (sizeof(T) == 4) {
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2, %3;\n" ::"r"(s), "l"(gmem),
                     "r"(nbytes), "l"(pol)
                     : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2, %3;\n" ::"r"(s), "l"(gmem),
                     "r"(nbytes), "l"(pol)
                     : "memory");
    }
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Explicitly rounded multiply / fused multiply-add, so that every kernel that
// evaluates the same interpolant gets bit-identical results regardless of
// the compiler's contraction choices.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Linear interpolation wl*a + wr*b (the weights of an odd node's two coarse
// neighbours), always evaluated as fma(wl, a, wr*b).
template <typename T>
__device__ __forceinline__ T lerp2(T wl, T a, T wr, T b)
{
    return fma_rn(wl, a, mul_rn(wr, b));
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialization attribute (launch_pdl) is scheduled as the blocks of
// its predecessor on the stream exit, so its launch and first blocks overlap
// the predecessor's last wave: pdl_wait() returns once the predecessor has
// completed and its memory operations are visible (at once for a kernel
// launched without the attribute), so every such kernel calls it before
// touching memory its predecessor writes or reads.  (An explicit early
// trigger, which lets the successor's blocks wait on the SMs from the start,
// measured slower.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Streaming (evict-first) global store for data that is not read again soon.
template <typename T>
__device__ __forceinline__ void st_stream(T *p, T v)
{
    __stcs(p, v);
}

}  // namespace mg
