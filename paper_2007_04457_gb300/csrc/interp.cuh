// interp.cuh -- the element-wise level kernels, on a (x-chunk, row, plane)
// grid of small threads so every kernel runs at full occupancy with many
// independent loads in flight; interpolation corners are re-read from L1.
//
// k_coef (decomposition, after the coarser levels are done): every node of
//   N_l \ N_{l-1} receives its coefficient u - Pi_{l-1} u, recomputed from the
//   untouched level array with the same explicitly rounded interpolation as
//   the restriction kernel (so it is bit-identical to the C that entered the
//   load vector).  The N_{l-1} nodes are rewritten with their own (unchanged)
//   value, which keeps the written sectors whole and cannot race with the
//   threads that read them as corners.
// k_scatter: the N_{l-1} nodes then receive the final coarse values V
//   (Fig. 3: each node keeps the value of the coarsest level it belongs to).
// k_interp (recomposition, Section II-A): the even nodes receive the
//   corrected coarse nodal values V, every other node its coefficient plus
//   the multilinear interpolant of V.
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

// Each thread of k_coef / k_interp handles the 4 consecutive nodes
// x0 .. x0+3 (x0 = 4t) of one row, so the even corner columns x0, x0+2,
// x0+4 of every row it interpolates from are loaded once for four nodes.
template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kRowThreads) k_coef(PlaceParams p)
{
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2;
    const NodeIter it = node_iter();
    const int64_t x0 = 4 * it.x;
    if (x0 >= n2) return;
    const int nk = (int)min64(4, n2 - x0);
    const bool has2 = x0 + 2 < n2, has4 = x0 + 4 < n2;
    const T wa1 = (x0 + 1 < n2 - 1) ? w2[2 * (x0 + 1)] : T(0), wb1 = (x0 + 1 < n2 - 1) ? w2[2 * (x0 + 1) + 1] : T(0);
    const T wa3 = (x0 + 3 < n2 - 1) ? w2[2 * (x0 + 3)] : T(0), wb3 = (x0 + 3 < n2 - 1) ? w2[2 * (x0 + 3) + 1] : T(0);
    // x-interpolant of row r at the four nodes, from its even columns
    auto X4 = [&](const T *r, T (&o)[4]) {
        const T e0 = r[x0], e2 = has2 ? r[x0 + 2] : T(0), e4 = has4 ? r[x0 + 4] : T(0);
        o[0] = e0;
        o[1] = lerp2(wa1, e0, wb1, e2);
        o[2] = e2;
        o[3] = lerp2(wa3, e2, wb3, e4);
    };
    for (int64_t z = it.z0; z < n0; z += it.zstep) {
        const bool oz = HZ && (z & 1);
        const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
        const int64_t za = oz ? z - 1 : z, zb = oz ? z + 1 : z;
        for (int64_t y = it.y0; y < n1; y += it.ystep) {
            const bool oy = HY && (y & 1);
            const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
            const int64_t ya = oy ? y - 1 : y, yb = oy ? y + 1 : y;
            T *arow = A + (z * n1 + y) * n2;
            T u[4], I[4], t[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) u[k] = (k < nk) ? arow[x0 + k] : T(0);
            X4(A + (za * n1 + ya) * n2, I);
            if (oy) {
                X4(A + (za * n1 + yb) * n2, t);
#pragma unroll
                for (int k = 0; k < 4; ++k) I[k] = lerp2(wya, I[k], wyb, t[k]);
            }
            if (oz) {
                T b[4];
                X4(A + (zb * n1 + ya) * n2, b);
                if (oy) {
                    X4(A + (zb * n1 + yb) * n2, t);
#pragma unroll
                    for (int k = 0; k < 4; ++k) b[k] = lerp2(wya, b[k], wyb, t[k]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) I[k] = lerp2(wza, I[k], wzb, b[k]);
            }
            const bool eo = !oy && !oz;  // even row: even columns are coarse nodes
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k < nk) {
                    const T out = (eo && !(k & 1)) ? u[k] : sub_rn(u[k], I[k]);
                    __stcg(arow + x0 + k, out);  // opaque store: coarse nodes are rewritten unchanged
                }
            }
        }
    }
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

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kRowThreads) k_interp(PlaceParams p)
{
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2, m1 = p.m1, m2 = p.m2;
    const NodeIter it = node_iter();
    const int64_t x0 = 4 * it.x;
    if (x0 >= n2) return;
    const int nk = (int)min64(4, n2 - x0);
    const int64_t X0 = x0 >> 1;
    const bool has1 = X0 + 1 < m2, has2 = X0 + 2 < m2;
    const T wa1 = (x0 + 1 < n2 - 1) ? w2[2 * (x0 + 1)] : T(0), wb1 = (x0 + 1 < n2 - 1) ? w2[2 * (x0 + 1) + 1] : T(0);
    const T wa3 = (x0 + 3 < n2 - 1) ? w2[2 * (x0 + 3)] : T(0), wb3 = (x0 + 3 < n2 - 1) ? w2[2 * (x0 + 3) + 1] : T(0);
    auto X4 = [&](const TW *r, T (&o)[4]) {
        const T v0 = static_cast<T>(r[X0]);
        const T v1 = has1 ? static_cast<T>(r[X0 + 1]) : T(0);
        const T v2 = has2 ? static_cast<T>(r[X0 + 2]) : T(0);
        o[0] = v0;
        o[1] = lerp2(wa1, v0, wb1, v1);
        o[2] = v1;
        o[3] = lerp2(wa3, v1, wb3, v2);
    };
    for (int64_t z = it.z0; z < n0; z += it.zstep) {
        const bool oz = HZ && (z & 1);
        const int64_t Za = HZ ? (z >> 1) : 0, Zb = Za + (oz ? 1 : 0);
        const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
        for (int64_t y = it.y0; y < n1; y += it.ystep) {
            const bool oy = HY && (y & 1);
            const int64_t Ya = HY ? (y >> 1) : 0, Yb = Ya + (oy ? 1 : 0);
            const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
            T *arow = A + (z * n1 + y) * n2;
            T c[4], I[4], t[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = (k < nk) ? arow[x0 + k] : T(0);
            X4(V + (Za * m1 + Ya) * m2, I);
            if (oy) {
                X4(V + (Za * m1 + Yb) * m2, t);
#pragma unroll
                for (int k = 0; k < 4; ++k) I[k] = lerp2(wya, I[k], wyb, t[k]);
            }
            if (oz) {
                T b[4];
                X4(V + (Zb * m1 + Ya) * m2, b);
                if (oy) {
                    X4(V + (Zb * m1 + Yb) * m2, t);
#pragma unroll
                    for (int k = 0; k < 4; ++k) b[k] = lerp2(wya, b[k], wyb, t[k]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) I[k] = lerp2(wza, I[k], wzb, b[k]);
            }
            const bool eo = !oy && !oz;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < nk) arow[x0 + k] = (eo && !(k & 1)) ? I[k] : add_rn(c[k], I[k]);
        }
    }
}

}  // namespace mg
