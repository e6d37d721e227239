// quant.cuh -- uniform quantization of the coefficient classes of a
// decomposed field and its inverse (the quantization and de-quantization
// steps that the paper's lossy-compression showcase runs on the GPU after the
// decomposition, Section V-B).
//
// Class of node (z, y, x) in the in-place layout of L levels (Fig. 3): the
// smallest l whose node set (indices multiple of 2^(L-l) in every dimension)
// holds it, i.e. max over dimensions of max(0, L - trailing_zeros(index))
// (index 0 counts as class 0).  Code: sign(c) floor(|c| (1 / bin_k) + 1/2)
// in the field's precision (one rounded product, one rounded addition),
// saturating at +-(2^31 - 1); de-quantized value: code x bin_k.  One warp per
// row of the field, coalesced 4- or 8-byte accesses.
#pragma once

#include <climits>

#include "common.cuh"

namespace mg {

constexpr int kQuantWarps = 8;
constexpr int kQuantMaxClasses = 32;

template <typename T>
struct QuantParams {
    const T *c;        // quantize: the decomposed field
    int32_t *q;        // quantize: codes out
    const int32_t *qi; // de-quantize: codes in
    T *d;              // de-quantize: the field out
    int64_t n0, n1, n2;
    int L;
    T inv[kQuantMaxClasses];   // 1 / bin_k rounded to T
    T bin[kQuantMaxClasses];   // bin_k rounded to T
};

__device__ __forceinline__ int index_class(int64_t i, int L)
{
    if (i == 0) return 0;
    const int tz = __ffsll((long long)i) - 1;
    return tz >= L ? 0 : L - tz;
}

template <typename T>
__device__ __forceinline__ int32_t quantize_one(T c, T inv)
{
    const T m = mul_rn(c < T(0) ? -c : c, inv);
    const T r = floor(add_rn(m, T(0.5)));
    const int32_t code = (r >= T(2147483648.0)) ? INT_MAX : (int32_t)r;
    return c < T(0) ? -code : code;
}

// MODE 0: quantize c -> q; MODE 1: de-quantize qi -> d
template <typename T, int MODE>
__global__ void __launch_bounds__(32 * kQuantWarps) k_quant(QuantParams<T> p)
{
    const int lane = threadIdx.x & 31;
    const int64_t rows = p.n0 * p.n1;
    for (int64_t row = (int64_t)blockIdx.x * kQuantWarps + (threadIdx.x >> 5); row < rows;
         row += (int64_t)gridDim.x * kQuantWarps) {
        const int64_t z = row / p.n1, y = row - z * p.n1;
        const int rc = max(index_class(z, p.L), index_class(y, p.L));
        const int64_t base = row * p.n2;
        for (int64_t x0 = 0; x0 < p.n2; x0 += 128) {
            T v[4];
            int32_t qv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t x = x0 + 32 * k + lane;
                if (x < p.n2) {
                    if constexpr (MODE == 0) v[k] = p.c[base + x];
                    else qv[k] = p.qi[base + x];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t x = x0 + 32 * k + lane;
                if (x < p.n2) {
                    const int cls = max(rc, index_class(x, p.L));
                    if constexpr (MODE == 0) p.q[base + x] = quantize_one(v[k], p.inv[cls]);
                    else p.d[base + x] = mul_rn(static_cast<T>(qv[k]), p.bin[cls]);
                }
            }
        }
    }
}

}  // namespace mg
