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
// one warp 32 nodes per step.  Per step every lane first forms one coarse
// column of the row's interpolant in dims 0 and 1 (four loads of V, which
// stays in L2: each level-k row serves up to (2^(D+1) - 1)^2 finest rows,
// visited close together), then takes the two columns that bracket its node
// from their lanes by shuffles: with D >= 1, 32 consecutive nodes span at
// most 17 coarse columns.  A node on N_k gets weight 0 on its right
// neighbour, so its value is copied exactly.
template <typename T, typename TW>
__global__ void __launch_bounds__(kProlongThreads) k_prolong(ProlongParams p)
{
    T *__restrict__ out = static_cast<T *>(p.out);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const TW *__restrict__ w0 = static_cast<const TW *>(p.w0);
    const TW *__restrict__ w1 = static_cast<const TW *>(p.w1);
    const TW *__restrict__ w2 = static_cast<const TW *>(p.w2);
    const int lane = threadIdx.x & 31;
    const int sh = p.shift;
    const int64_t nseg = (p.n2 + p.seg - 1) / p.seg;
    const int64_t items = (int64_t)p.n0 * p.n1 * nseg;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
        const int64_t r = it / nseg;
        const int xs = (int)(it - r * nseg) * p.seg;
        const int xe = min(xs + p.seg, p.n2);
        const int i0 = (int)(r / p.n1), i1 = (int)(r - (int64_t)i0 * p.n1);
        const int c0 = i0 >> sh, c1 = i1 >> sh;
        const int c0b = min(c0 + 1, p.m0 - 1), c1b = min(c1 + 1, p.m1 - 1);
        const TW a0 = w0[i0], a1 = w1[i1];
        const TW *r00 = V + ((int64_t)c0 * p.m1 + c1) * p.m2;
        const TW *r01 = V + ((int64_t)c0 * p.m1 + c1b) * p.m2;
        const TW *r10 = V + ((int64_t)c0b * p.m1 + c1) * p.m2;
        const TW *r11 = V + ((int64_t)c0b * p.m1 + c1b) * p.m2;
        T *orow = out + r * p.n2;
        for (int x0 = xs; x0 < xe; x0 += 32) {
            const int cb = x0 >> sh;
            const int cc = min(cb + lane, p.m2 - 1);
            const TW v00 = r00[cc], v01 = r01[cc], v10 = r10[cc], v11 = r11[cc];
            const TW t0 = v00 + a1 * (v01 - v00);
            const TW t1 = v10 + a1 * (v11 - v10);
            const TW col = t0 + a0 * (t1 - t0);
            const int i2 = min(x0 + lane, p.n2 - 1);
            const int cl = i2 >> sh;
            const int cr = min(cl + 1, p.m2 - 1);
            const TW vl = __shfl_sync(0xffffffffu, col, cl - cb);
            const TW vr = __shfl_sync(0xffffffffu, col, cr - cb);
            if (x0 + lane < xe) {
                const TW a2 = w2[i2];
                orow[i2] = static_cast<T>(vl + a2 * (vr - vl));
            }
        }
    }
}

}  // namespace mg
