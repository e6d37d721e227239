// interp.cuh -- the element-wise level kernels: one thread per fine node on
// a (x-chunk, row, plane) grid, so every kernel runs at full occupancy with
// independent loads in flight; the interpolation corners are re-read from L1.
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
    const int64_t x = it.x;
    if (x >= n2) return;
    const bool ox = (x & 1);
    const T wxa = ox ? w2[2 * x] : T(0), wxb = ox ? w2[2 * x + 1] : T(0);
    const int64_t xl = ox ? x - 1 : x, xr = ox ? x + 1 : x;
    for (int64_t z = it.z0; z < n0; z += it.zstep) {
        const bool oz = HZ && (z & 1);
        const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
        const int64_t za = oz ? z - 1 : z, zb = oz ? z + 1 : z;
        for (int64_t y = it.y0; y < n1; y += it.ystep) {
            const bool oy = HY && (y & 1);
            T *a = A + (z * n1 + y) * n2 + x;
            const T u = *a;
            if (!ox && !oy && !oz) {
                __stcg(a, u);  // coarse node: rewritten unchanged (opaque store keeps the
                continue;      // sector whole); its final value comes from k_scatter
            }
            const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
            const int64_t ya = oy ? y - 1 : y, yb = oy ? y + 1 : y;
            auto X = [&](int64_t zz, int64_t yy) -> T {
                const T *r = A + (zz * n1 + yy) * n2;
                return ox ? lerp2(wxa, r[xl], wxb, r[xr]) : r[x];
            };
            const T ia = oy ? lerp2(wya, X(za, ya), wyb, X(za, yb)) : X(za, ya);
            T iv = ia;
            if (oz) {
                const T ib = oy ? lerp2(wya, X(zb, ya), wyb, X(zb, yb)) : X(zb, ya);
                iv = lerp2(wza, ia, wzb, ib);
            }
            *a = sub_rn(u, iv);
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
    const int64_t x = it.x;
    if (x >= n2) return;
    const bool ox = (x & 1);
    const int64_t Xa = x >> 1, Xb = ox ? Xa + 1 : Xa;
    const T wxa = ox ? w2[2 * x] : T(0), wxb = ox ? w2[2 * x + 1] : T(0);
    for (int64_t z = it.z0; z < n0; z += it.zstep) {
        const bool oz = HZ && (z & 1);
        const int64_t Za = HZ ? (z >> 1) : 0, Zb = Za + (oz ? 1 : 0);
        const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
        for (int64_t y = it.y0; y < n1; y += it.ystep) {
            const bool oy = HY && (y & 1);
            const int64_t Ya = HY ? (y >> 1) : 0, Yb = Ya + (oy ? 1 : 0);
            T *a = A + (z * n1 + y) * n2 + x;
            auto X = [&](int64_t ZZ, int64_t YY) -> T {
                const TW *r = V + (ZZ * m1 + YY) * m2;
                return ox ? lerp2(wxa, static_cast<T>(r[Xa]), wxb, static_cast<T>(r[Xb])) : static_cast<T>(r[Xa]);
            };
            if (!ox && !oy && !oz) {
                *a = X(Za, Ya);
                continue;
            }
            const T c = *a;
            const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
            const T ia = oy ? lerp2(wya, X(Za, Ya), wyb, X(Za, Yb)) : X(Za, Ya);
            T iv = ia;
            if (oz) {
                const T ib = oy ? lerp2(wya, X(Zb, Ya), wyb, X(Zb, Yb)) : X(Zb, Ya);
                iv = lerp2(wza, ia, wzb, ib);
            }
            *a = add_rn(c, iv);
        }
    }
}

}  // namespace mg
