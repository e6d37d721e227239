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
constexpr int kProlongRows = 64;   // finest rows (dim 1) per work item

// Work item = a strip of 32 finest columns x kProlongRows finest rows of one
// plane i0, handled by one warp walking down the rows.  Lane L loads, per
// level-k row, the dim-0 interpolant of coarse column (first column of the
// strip >> D) + L (two loads of V; with D >= 1 a strip spans at most 17
// coarse columns); the warp keeps the two level-k rows that bracket its
// current row in registers and prefetches the next one, so a finest row
// costs one interpolation in dim 1, two shuffles (the coarse columns left and
// right of the lane's node), one in dim 2 and a store.  Consecutive warps
// take neighbouring strips of the same rows, sharing their coarse rows in L1.
// A node on N_k gets weight 0 on every right neighbour, so its value is
// copied exactly.  The launch (launch_impl.cuh) sizes the grid to one wave
// of resident blocks; the loop below covers every item whatever the grid.
template <typename T, typename TW>
__global__ void __launch_bounds__(kProlongThreads, sizeof(TW) == 4 ? kProlongBlocksPerSm : 5) k_prolong(ProlongParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    T *__restrict__ out = static_cast<T *>(p.out);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const TW *__restrict__ w0 = static_cast<const TW *>(p.w0);
    const TW *__restrict__ w1 = static_cast<const TW *>(p.w1);
    const TW *__restrict__ w2 = static_cast<const TW *>(p.w2);
    const int lane = threadIdx.x & 31;
    const int sh = p.shift, n1 = p.n1, n2 = p.n2, m1 = p.m1, m2 = p.m2;
    const int64_t nstrip = (n2 + 31) / 32;
    const int64_t per_plane = nstrip * ((n1 + kProlongRows - 1) / kProlongRows);
    const int64_t items = (int64_t)p.n0 * per_plane;
    const int64_t plane_m = (int64_t)m1 * m2;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
        const int i0 = (int)(it / per_plane);
        const int64_t rem = it - (int64_t)i0 * per_plane;
        const int ch = (int)(rem / nstrip);
        const int xs = (int)(rem - (int64_t)ch * nstrip) * 32;
        const int x = xs + lane;
        const int xc = min(x, n2 - 1);
        const int cb = xs >> sh;
        const int sl = (xc >> sh) - cb;                          // 0 .. 15
        const int sr = min((xc >> sh) + 1, m2 - 1) - cb;         // 0 .. 16
        const TW a2 = w2[xc];
        const int c0 = i0 >> sh, c0b = min(c0 + 1, p.m0 - 1);
        const TW a0 = w0[i0];
        const int cc = min(cb + lane, m2 - 1);
        const TW *P0 = V + (int64_t)c0 * plane_m + cc;
        const TW *P1 = V + (int64_t)c0b * plane_m + cc;
        const int ys = ch * kProlongRows, ye = min(ys + kProlongRows, n1);
        int c1 = ys >> sh;
        int cn = min(c1 + 1, m1 - 1);
        const TW l0 = P0[(int64_t)c1 * m2], l1 = P1[(int64_t)c1 * m2];
        const TW h0 = P0[(int64_t)cn * m2], h1 = P1[(int64_t)cn * m2];
        cn = min(c1 + 2, m1 - 1);
        TW q0 = P0[(int64_t)cn * m2], q1 = P1[(int64_t)cn * m2];   // the level-k row after `hi`
        TW lo = l0 + a0 * (l1 - l0);
        TW hi = h0 + a0 * (h1 - h0);
        int64_t idx = ((int64_t)i0 * n1 + ys) * n2 + x;
        for (int y = ys; y < ye; ++y, idx += n2) {
            if ((y >> sh) != c1) {  // the warp moves on to the next level-k row
                c1 = y >> sh;
                lo = hi;
                hi = q0 + a0 * (q1 - q0);
                cn = min(c1 + 2, m1 - 1);
                q0 = P0[(int64_t)cn * m2];
                q1 = P1[(int64_t)cn * m2];
            }
            const TW a1 = w1[y];
            const TW t = lo + a1 * (hi - lo);
            const TW vl = __shfl_sync(0xffffffffu, t, sl);
            const TW vr = __shfl_sync(0xffffffffu, t, sr);
            if (x < n2) out[idx] = static_cast<T>(vl + a2 * (vr - vl));
        }
    }
}

}  // namespace mg
