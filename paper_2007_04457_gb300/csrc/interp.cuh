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

// k_coef / k_interp: a warp takes a 128-node segment of one row; lane L
// handles the nodes base + L + 32k (k < 4), so every load is one coalesced
// 128-byte access.  An odd node's even neighbours x-1 and x+1 come from the
// adjacent lanes by shuffle (lane 31 takes x+1 from lane 0 of the next
// group, or loads it after the last group).
constexpr int kSegChunks = 4;
constexpr int kSeg = 32 * kSegChunks;

template <typename T>
__device__ __forceinline__ void odd_neighbours(const T (&e)[kSegChunks], T extra, int lane, T (&left)[kSegChunks],
                                               T (&right)[kSegChunks])
{
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k) {
        left[k] = __shfl_up_sync(0xffffffffu, e[k], 1);
        const T dn = __shfl_down_sync(0xffffffffu, e[k], 1);
        const T nx = (k + 1 < kSegChunks) ? __shfl_sync(0xffffffffu, e[(k + 1) % kSegChunks], 0) : extra;
        right[k] = (lane == 31) ? nx : dn;
    }
}

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kRowThreads) k_coef(PlaceParams p)
{
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2;
    const int lane = threadIdx.x & 31;
    const int64_t segs = (n2 + kSeg - 1) / kSeg;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (wid >= n0 * n1 * segs) return;  // whole warps only
    const int64_t row = wid / segs, base = (wid - row * segs) * kSeg;
    const int64_t z = row / n1, y = row - (row / n1) * n1;
    const bool ox = lane & 1;
    const bool oz = HZ && (z & 1), oy = HY && (y & 1);
    const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
    const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
    const int64_t za = oz ? z - 1 : z, zb = oz ? z + 1 : z;
    const int64_t ya = oy ? y - 1 : y, yb = oy ? y + 1 : y;
    T wa[kSegChunks], wb[kSegChunks];
    bool valid[kSegChunks];
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k) {
        const int64_t x = base + lane + 32 * k;
        valid[k] = x < n2;
        const bool wok = ox && x < n2 - 1;
        wa[k] = wok ? w2[2 * x] : T(0);
        wb[k] = wok ? w2[2 * x + 1] : T(0);
    }
    const bool has_extra = base + kSeg < n2;
    // x-interpolant of row r at the lane's nodes (even nodes: the value itself)
    auto Xrow = [&](const T *r, T (&o)[kSegChunks]) {
        T e[kSegChunks], l[kSegChunks], rr[kSegChunks];
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) e[k] = valid[k] ? r[base + lane + 32 * k] : T(0);
        const T extra = has_extra ? r[base + kSeg] : T(0);
        odd_neighbours(e, extra, lane, l, rr);
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) o[k] = ox ? lerp2(wa[k], l[k], wb[k], rr[k]) : e[k];
    };
    T *arow = A + row * n2;
    T u[kSegChunks], I[kSegChunks], t[kSegChunks];
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k) u[k] = valid[k] ? arow[base + lane + 32 * k] : T(0);
    Xrow(A + (za * n1 + ya) * n2, I);
    if (oy) {
        Xrow(A + (za * n1 + yb) * n2, t);
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) I[k] = lerp2(wya, I[k], wyb, t[k]);
    }
    if (oz) {
        T b[kSegChunks];
        Xrow(A + (zb * n1 + ya) * n2, b);
        if (oy) {
            Xrow(A + (zb * n1 + yb) * n2, t);
#pragma unroll
            for (int k = 0; k < kSegChunks; ++k) b[k] = lerp2(wya, b[k], wyb, t[k]);
        }
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) I[k] = lerp2(wza, I[k], wzb, b[k]);
    }
    const bool coarse = !oy && !oz && !ox;  // even node of an even row: rewritten unchanged
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k)
        if (valid[k]) __stcg(arow + base + lane + 32 * k, coarse ? u[k] : sub_rn(u[k], I[k]));
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
    const int lane = threadIdx.x & 31;
    const int64_t segs = (n2 + kSeg - 1) / kSeg;
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (wid >= n0 * n1 * segs) return;  // whole warps only
    const int64_t row = wid / segs, base = (wid - row * segs) * kSeg;
    const int64_t z = row / n1, y = row - (row / n1) * n1;
    const bool ox = lane & 1;
    const bool oz = HZ && (z & 1), oy = HY && (y & 1);
    const int64_t Za = HZ ? (z >> 1) : 0, Zb = Za + (oz ? 1 : 0);
    const int64_t Ya = HY ? (y >> 1) : 0, Yb = Ya + (oy ? 1 : 0);
    const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
    const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
    T wa[kSegChunks], wb[kSegChunks];
    bool valid[kSegChunks];
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k) {
        const int64_t x = base + lane + 32 * k;
        valid[k] = x < n2;
        const bool wok = ox && x < n2 - 1;
        wa[k] = wok ? w2[2 * x] : T(0);
        wb[k] = wok ? w2[2 * x + 1] : T(0);
    }
    const bool has_extra = base + kSeg < n2;
    // x-interpolant of coarse row r at the lane's fine nodes: node x reads
    // V[x/2]; an odd node takes V[x/2 + 1] from the next lane
    auto Xrow = [&](const TW *r, T (&o)[kSegChunks]) {
        T e[kSegChunks], l[kSegChunks], rr[kSegChunks];
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) e[k] = valid[k] ? static_cast<T>(r[(base + lane + 32 * k) >> 1]) : T(0);
        const T extra = has_extra ? static_cast<T>(r[(base + kSeg) >> 1]) : T(0);
        odd_neighbours(e, extra, lane, l, rr);
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) o[k] = ox ? lerp2(wa[k], e[k], wb[k], rr[k]) : e[k];
        (void)l;
    };
    T *arow = A + row * n2;
    T c[kSegChunks], I[kSegChunks], t[kSegChunks];
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k) c[k] = valid[k] ? arow[base + lane + 32 * k] : T(0);
    Xrow(V + (Za * m1 + Ya) * m2, I);
    if (oy) {
        Xrow(V + (Za * m1 + Yb) * m2, t);
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) I[k] = lerp2(wya, I[k], wyb, t[k]);
    }
    if (oz) {
        T b[kSegChunks];
        Xrow(V + (Zb * m1 + Ya) * m2, b);
        if (oy) {
            Xrow(V + (Zb * m1 + Yb) * m2, t);
#pragma unroll
            for (int k = 0; k < kSegChunks; ++k) b[k] = lerp2(wya, b[k], wyb, t[k]);
        }
#pragma unroll
        for (int k = 0; k < kSegChunks; ++k) I[k] = lerp2(wza, I[k], wzb, b[k]);
    }
    const bool coarse = !oy && !oz && !ox;
#pragma unroll
    for (int k = 0; k < kSegChunks; ++k)
        if (valid[k]) arow[base + lane + 32 * k] = coarse ? I[k] : add_rn(c[k], I[k]);
}

}  // namespace mg
