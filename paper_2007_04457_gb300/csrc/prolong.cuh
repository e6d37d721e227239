// prolong.cuh -- finest-grid values of a level-k function: multilinear
// interpolation of the compact level-k values V (N_k, every 2^D-th node of
// each active dimension, D = L - k) onto every node of the finest grid.
//
// Recomposition from the first k+1 coefficient classes (Section I, Fig. 1;
// Section II-A, overall process) leaves the classes of levels k+1 .. L out:
// their coefficients are zero, so at those levels the load vector and the
// correction vanish and each recomposition step reduces to interpolation
// from the next coarser level.  Interpolating level by level and
// interpolating once from N_k give the same piecewise-multilinear function
// (linear interpolation reproduces linear functions), so one pass that only
// writes the finest array replaces D level steps.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kProlongThreads = 256;
constexpr int kProlongBlocksPerSm = 8;

// Work item = p.seg consecutive nodes of one finest row (i0, i1), handled by
// one warp 32 nodes per step, two steps per iteration with the loads of both
// issued first.  Per step every lane forms one coarse column of the row's
// interpolant in dims 0 and 1 (four loads of V, which stays in L2: each
// level-k row serves up to (2^(D+1) - 1)^2 finest rows, visited close
// together), then takes the two columns that bracket its node from their
// lanes by shuffles: with D >= 1, 32 consecutive nodes span at most 17
// coarse columns.  A node on N_k gets weight 0 on its right neighbour, so
// its value is copied exactly.
template <typename TW>
__device__ __forceinline__ TW prolong_col(const TW *r00, const TW *r01, const TW *r10, const TW *r11, int c,
                                          TW a0, TW a1)
{
    const TW v00 = r00[c], v01 = r01[c], v10 = r10[c], v11 = r11[c];
    const TW t0 = v00 + a1 * (v01 - v00);
    const TW t1 = v10 + a1 * (v11 - v10);
    return t0 + a0 * (t1 - t0);
}

template <typename T, typename TW>
__global__ void __launch_bounds__(kProlongThreads) k_prolong(ProlongParams p)
{
    T *__restrict__ out = static_cast<T *>(p.out);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const TW *__restrict__ w0 = static_cast<const TW *>(p.w0);
    const TW *__restrict__ w1 = static_cast<const TW *>(p.w1);
    const TW *__restrict__ w2 = static_cast<const TW *>(p.w2);
    const int lane = threadIdx.x & 31;
    const int sh = p.shift, n2 = p.n2, m2 = p.m2;
    const unsigned nseg = (unsigned)((n2 + p.seg - 1) / p.seg);
    const unsigned items = (unsigned)p.n0 * (unsigned)p.n1 * nseg;  // < 2^31 (host check)
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
        const unsigned r = it / nseg;
        const int xs = (int)(it - r * nseg) * p.seg;
        const int xe = min(xs + p.seg, n2);
        const int i0 = (int)(r / (unsigned)p.n1), i1 = (int)(r - (unsigned)i0 * (unsigned)p.n1);
        const int c0 = i0 >> sh, c1 = i1 >> sh;
        const int c0b = min(c0 + 1, p.m0 - 1), c1b = min(c1 + 1, p.m1 - 1);
        const TW a0 = w0[i0], a1 = w1[i1];
        const TW *r00 = V + ((int64_t)c0 * p.m1 + c1) * m2;
        const TW *r01 = V + ((int64_t)c0 * p.m1 + c1b) * m2;
        const TW *r10 = V + ((int64_t)c0b * p.m1 + c1) * m2;
        const TW *r11 = V + ((int64_t)c0b * p.m1 + c1b) * m2;
        T *orow = out + (int64_t)r * n2;
        for (int x0 = xs; x0 < xe; x0 += 64) {
            // second step of the pair: when it lies past the segment, its
            // indexes collapse onto the last node (in bounds, not stored)
            const int y0 = min(x0 + 32, n2 - 1);
            const int cbA = x0 >> sh, cbB = y0 >> sh;
            const int i2A = min(x0 + lane, n2 - 1), i2B = min(y0 + lane, n2 - 1);
            const TW colA = prolong_col(r00, r01, r10, r11, min(cbA + lane, m2 - 1), a0, a1);
            const TW colB = prolong_col(r00, r01, r10, r11, min(cbB + lane, m2 - 1), a0, a1);
            const TW a2A = w2[i2A], a2B = w2[i2B];
            const int clA = i2A >> sh, clB = i2B >> sh;
            const TW lA = __shfl_sync(0xffffffffu, colA, clA - cbA);
            const TW rA = __shfl_sync(0xffffffffu, colA, min(clA + 1, m2 - 1) - cbA);
            const TW lB = __shfl_sync(0xffffffffu, colB, clB - cbB);
            const TW rB = __shfl_sync(0xffffffffu, colB, min(clB + 1, m2 - 1) - cbB);
            if (x0 + lane < xe) orow[i2A] = static_cast<T>(lA + a2A * (rA - lA));
            if (x0 + 32 + lane < xe) orow[i2B] = static_cast<T>(lB + a2B * (rB - lB));
        }
    }
}

}  // namespace mg
