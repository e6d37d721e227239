// interp.cuh -- the two element-wise level kernels.
//
// k_place (decomposition, after the coarser levels are done): every node of
//   N_l \ N_{l-1} receives its coefficient u - Pi_{l-1} u, recomputed from the
//   untouched level array with the same explicitly rounded interpolation as
//   the restriction kernel (so it is bit-identical to the C that entered the
//   load vector), and the N_{l-1} nodes receive the final coarse values V
//   (Fig. 3: each node keeps the value of the coarsest level it belongs to).
//   Phase 0 handles the rows that are odd in dim 0 or dim 1: they only read
//   their own nodes and the N_{l-1} nodes of even rows, which phase 0 never
//   writes.  Phase 1 handles the even rows: a warp reads a batch of its row,
//   syncs, then writes it; an odd node's left neighbour is in the same batch
//   and its right neighbour in the same or the next, not yet written, batch.
// k_interp (recomposition, Section II-A): the even nodes receive the
//   corrected coarse nodal values V, every other node its coefficient plus
//   the multilinear interpolant of V.
//
// Both run one warp per grid row (fixed dims 0 and 1), lanes along the
// contiguous dimension; each lane handles kBatch nodes of the row at a time
// and issues all their loads before any arithmetic, so a warp keeps many
// independent loads in flight.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kRowThreads = 256;
constexpr int kBatch = 8;

template <typename T, typename TW, int ACT, int PHASE>
__global__ void __launch_bounds__(kRowThreads) k_place(PlaceParams p)
{
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int lane = threadIdx.x & 31;
    const int64_t n1 = p.n1, n2 = p.n2;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t wfirst = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);

    if constexpr (PHASE == 0) {
        const int64_t nrows = p.n0 * n1;
        for (int64_t row = wfirst; row < nrows; row += wstride) {
            const int64_t z = row / n1, y = row - (row / n1) * n1;
            const bool oz = HZ && (z & 1), oy = HY && (y & 1);
            if (!oz && !oy) continue;
            const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
            const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
            const int64_t za = oz ? z - 1 : z, zb = oz ? z + 1 : z;
            const int64_t ya = oy ? y - 1 : y, yb = oy ? y + 1 : y;
            const T *raa = A + (za * n1 + ya) * n2;
            const T *rab = A + (za * n1 + yb) * n2;
            const T *rba = A + (zb * n1 + ya) * n2;
            const T *rbb = A + (zb * n1 + yb) * n2;
            T *arow = A + row * n2;
            for (int64_t base = 0; base < n2; base += 32 * kBatch) {
                T u[kBatch], iv[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const int64_t x = base + lane + 32 * k;
                    u[k] = T(0);
                    iv[k] = T(0);
                    if (x < n2) {
                        const bool ox = (x & 1);
                        const T wxa = ox ? w2[2 * x] : T(0), wxb = ox ? w2[2 * x + 1] : T(0);
                        const int64_t xl = ox ? x - 1 : x, xr = ox ? x + 1 : x;
                        auto X = [&](const T *r) -> T { return ox ? lerp2(wxa, r[xl], wxb, r[xr]) : r[x]; };
                        u[k] = __ldcs(arow + x);
                        const T ia = oy ? lerp2(wya, X(raa), wyb, X(rab)) : X(raa);
                        if (oz) {
                            const T ib = oy ? lerp2(wya, X(rba), wyb, X(rbb)) : X(rba);
                            iv[k] = lerp2(wza, ia, wzb, ib);
                        } else {
                            iv[k] = ia;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const int64_t x = base + lane + 32 * k;
                    if (x < n2) __stcs(arow + x, sub_rn(u[k], iv[k]));
                }
            }
        }
    } else {
        const int64_t nrows = p.m0 * p.m1;
        for (int64_t r = wfirst; r < nrows; r += wstride) {
            const int64_t Z = r / p.m1, Y = r - (r / p.m1) * p.m1;
            const int64_t z = HZ ? 2 * Z : 0, y = HY ? 2 * Y : 0;
            T *arow = A + (z * n1 + y) * n2;
            const TW *vrow = V + r * p.m2;
            for (int64_t base = 0; base < n2; base += 32 * kBatch) {
                T out[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const int64_t x = base + lane + 32 * k;
                    out[k] = T(0);
                    if (x < n2) {
                        if (x & 1)
                            out[k] = sub_rn(arow[x], lerp2(w2[2 * x], arow[x - 1], w2[2 * x + 1], arow[x + 1]));
                        else
                            out[k] = static_cast<T>(vrow[x >> 1]);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const int64_t x = base + lane + 32 * k;
                    if (x < n2) arow[x] = out[k];
                }
                __syncwarp();
            }
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
    const int lane = threadIdx.x & 31;
    const int64_t nrows = p.n0 * p.n1;
    const int64_t n2 = p.n2;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); row < nrows;
         row += wstride) {
        const int64_t z = row / p.n1, y = row - (row / p.n1) * p.n1;
        const bool oz = HZ && (z & 1), oy = HY && (y & 1);
        const int64_t Za = HZ ? (z >> 1) : 0, Ya = HY ? (y >> 1) : 0;
        const int64_t Zb = Za + (oz ? 1 : 0), Yb = Ya + (oy ? 1 : 0);
        const T wza = oz ? w0[2 * z] : T(0), wzb = oz ? w0[2 * z + 1] : T(0);
        const T wya = oy ? w1[2 * y] : T(0), wyb = oy ? w1[2 * y + 1] : T(0);
        const TW *vaa = V + (Za * p.m1 + Ya) * p.m2;
        const TW *vab = V + (Za * p.m1 + Yb) * p.m2;
        const TW *vba = V + (Zb * p.m1 + Ya) * p.m2;
        const TW *vbb = V + (Zb * p.m1 + Yb) * p.m2;
        T *arow = A + row * n2;
        for (int64_t base = 0; base < n2; base += 32 * kBatch) {
            T out[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int64_t x = base + lane + 32 * k;
                out[k] = T(0);
                if (x < n2) {
                    const int64_t Xa = x >> 1;
                    const bool ox = (x & 1);
                    const int64_t Xb = ox ? Xa + 1 : Xa;
                    const T wxa = ox ? w2[2 * x] : T(0), wxb = ox ? w2[2 * x + 1] : T(0);
                    auto X = [&](const TW *r) -> T {
                        return ox ? lerp2(wxa, static_cast<T>(r[Xa]), wxb, static_cast<T>(r[Xb]))
                                  : static_cast<T>(r[Xa]);
                    };
                    const T c = __ldcs(arow + x);
                    const T ia = oy ? lerp2(wya, X(vaa), wyb, X(vab)) : X(vaa);
                    T iv = ia;
                    if (oz) {
                        const T ib = oy ? lerp2(wya, X(vba), wyb, X(vbb)) : X(vba);
                        iv = lerp2(wza, ia, wzb, ib);
                    }
                    out[k] = (!ox && !oy && !oz) ? iv : add_rn(c, iv);
                }
            }
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int64_t x = base + lane + 32 * k;
                if (x < n2) __stcs(arow + x, out[k]);
            }
        }
    }
}

}  // namespace mg
