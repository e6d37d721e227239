// solve.cuh -- batched tridiagonal solves M_{l-1} z = f along one dimension
// of a compact coarse array (Section III-A-3: the correction solver, one
// Thomas solve per line).
//
// M_{l-1} is the same for every line of a dimension, so its LU factors are
// tabulated once per (level, dimension): forward y_i = f_i - a_i y_{i-1},
// backward z_i = inv_i y_i - q_i z_{i+1}.  Both sweeps are first-order linear
// recurrences.
//
// k_solve_panel: a block takes a panel of `lpb` lines (<= 32, one lane per
// line) and stages it in shared memory with cp.async: along a non-contiguous
// dimension the lines of a panel are adjacent in memory, so each node index
// of the panel is one coalesced row; along the contiguous dimension the panel
// is one contiguous block.  Each of the `nw` warps then owns a chunk of every
// line: it runs the recurrence over its chunk from a zero carry while
// accumulating the product of the multipliers, the chunk carries are
// composed through shared memory, and each chunk re-runs with its true
// carry.  The result goes back to F (or is added to / subtracted from V for
// the last dimension) with the same coalesced pattern.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

template <typename TW>
__device__ __forceinline__ void chunk_solve_smem(TW *row, const TW *fac, int s, int len, int w, int nw,
                                                 TW *carry_a, TW *carry_b, int lane)
{
    // forward: local run from zero carry, product of (-a_i)
    TW y = TW(0), pr = TW(1);
    for (int j = 0; j < len; ++j) {
        const TW a = fac[3 * (s + j)];
        y = row[s + j] - a * y;
        pr = -a * pr;
    }
    carry_a[w * 32 + lane] = y;
    carry_b[w * 32 + lane] = pr;
    __syncthreads();
    TW c = TW(0);
    for (int k = 0; k < w; ++k) c = carry_a[k * 32 + lane] + carry_b[k * 32 + lane] * c;
    __syncthreads();
    y = c;
    for (int j = 0; j < len; ++j) {
        y = row[s + j] - fac[3 * (s + j)] * y;
        row[s + j] = y;
    }
    // backward: z_i = inv_i y_i - q_i z_{i+1}, local run from zero carry
    TW z = TW(0);
    pr = TW(1);
    for (int j = len - 1; j >= 0; --j) {
        const TW inv = fac[3 * (s + j) + 1], q = fac[3 * (s + j) + 2];
        z = inv * row[s + j] - q * z;
        pr = -q * pr;
    }
    carry_a[w * 32 + lane] = z;
    carry_b[w * 32 + lane] = pr;
    __syncthreads();
    c = TW(0);
    for (int k = nw - 1; k > w; --k) c = carry_a[k * 32 + lane] + carry_b[k * 32 + lane] * c;
    z = c;
    for (int j = len - 1; j >= 0; --j) {
        z = fac[3 * (s + j) + 1] * row[s + j] - fac[3 * (s + j) + 2] * z;
        row[s + j] = z;
    }
}

// The same on a chunk held in registers (CH >= len): one shared-memory read
// and one write per node instead of four passes over shared memory.
template <typename TW, int CH>
__device__ __forceinline__ void chunk_solve_reg(TW *row, const TW *fac, int s, int len, int w, int nw,
                                                TW *carry_a, TW *carry_b, int lane)
{
    TW r[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) r[j] = (j < len) ? row[s + j] : TW(0);
    TW y = TW(0), pr = TW(1);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        if (j < len) {
            const TW a = fac[3 * (s + j)];
            y = r[j] - a * y;
            pr = -a * pr;
        }
    }
    carry_a[w * 32 + lane] = y;
    carry_b[w * 32 + lane] = pr;
    __syncthreads();
    TW c = TW(0);
    for (int k = 0; k < w; ++k) c = carry_a[k * 32 + lane] + carry_b[k * 32 + lane] * c;
    __syncthreads();
    y = c;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        if (j < len) {
            y = r[j] - fac[3 * (s + j)] * y;
            r[j] = y;
        }
    }
    TW z = TW(0);
    pr = TW(1);
#pragma unroll
    for (int j = CH - 1; j >= 0; --j) {
        if (j < len) {
            const TW inv = fac[3 * (s + j) + 1], q = fac[3 * (s + j) + 2];
            z = inv * r[j] - q * z;
            pr = -q * pr;
        }
    }
    carry_a[w * 32 + lane] = z;
    carry_b[w * 32 + lane] = pr;
    __syncthreads();
    c = TW(0);
    for (int k = nw - 1; k > w; --k) c = carry_a[k * 32 + lane] + carry_b[k * 32 + lane] * c;
    z = c;
#pragma unroll
    for (int j = CH - 1; j >= 0; --j) {
        if (j < len) {
            z = fac[3 * (s + j) + 1] * r[j] - fac[3 * (s + j) + 2] * z;
            r[j] = z;
        }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j)
        if (j < len) row[s + j] = r[j];
}

// Shared memory of k_solve_panel, in elements of TW.
inline size_t solve_panel_elems(int m, int lpb)
{
    return 2 * 32 * 32 + 3 * (size_t)m + 1 + (size_t)lpb * (size_t)(m | 1);
}

// CH > 0: chunks of at most CH nodes held in registers (at most 18 warps per
// block); CH = 0: chunks of any length solved in shared memory.
constexpr int kSolveRegWarps = 18;

template <typename TW, int CH>
__global__ void __launch_bounds__(CH > 0 ? 32 * kSolveRegWarps : 1024, 2) k_solve_panel(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *carry_a = reinterpret_cast<TW *>(smem_raw);
    TW *carry_b = carry_a + 32 * 32;
    TW *sfac = carry_b + 32 * 32;   // 3 m factors
    TW *tile = sfac + 3 * p.m + 1;  // lpb lines, pitch m | 1
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *fac = static_cast<const TW *>(p.fac);
    const int lane = threadIdx.x, w = threadIdx.y, nw = p.nw;
    const int tid = w * 32 + lane, nthr = 32 * nw;
    const int m = p.m, pitch = m | 1, lpb = p.lpb;
    const int64_t inner = p.inner, stride = p.stride;
    const bool contiguous = (inner == 1);
    const int chunk = p.chunk;
    const int s = w * chunk;
    const int len = max(0, min(chunk, m - s));

    for (int i = tid; i < 3 * m; i += nthr) sfac[i] = fac[i];

    for (int64_t panel = blockIdx.x; panel * lpb < p.nlines; panel += gridDim.x) {
        const int64_t line0 = panel * lpb;
        const int nl = (int)min64(lpb, p.nlines - line0);
        const int64_t myline = line0 + min(lane, nl - 1);
        const int64_t b_lane = myline / inner * (inner * m) + myline % inner;

        // stage the panel
        const TW *in = p.src ? static_cast<const TW *>(p.src) : F;
        if (contiguous) {
            const TW *src = in + line0 * m;
            int l = tid / m, i = tid - (tid / m) * m;
            const int step_l = nthr / m, step_i = nthr - (nthr / m) * m;
            for (int e = tid; e < nl * m; e += nthr) {
                cp_async_elem(tile + l * pitch + i, src + e, true);
                l += step_l;
                i += step_i;
                if (i >= m) { i -= m; ++l; }
            }
        } else if (lane < nl) {
            for (int i = w; i < m; i += nw) cp_async_elem(tile + lane * pitch + i, in + b_lane + (int64_t)i * stride, true);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();

        if constexpr (CH > 0)
            chunk_solve_reg<TW, CH>(tile + lane * pitch, sfac, s, len, w, nw, carry_a, carry_b, lane);
        else
            chunk_solve_smem<TW>(tile + lane * pitch, sfac, s, len, w, nw, carry_a, carry_b, lane);
        __syncthreads();

        // write back
        TW *dst = (p.vmode == 0) ? F : V;
        const TW sg = (p.vmode == 2) ? TW(-1) : TW(1);
        if (contiguous) {
            TW *d = dst + line0 * m;
            int l = tid / m, i = tid - (tid / m) * m;
            const int step_l = nthr / m, step_i = nthr - (nthr / m) * m;
            for (int e = tid; e < nl * m; e += nthr) {
                const TW r = tile[l * pitch + i];
                d[e] = (p.vmode == 0) ? r : d[e] + sg * r;
                l += step_l;
                i += step_i;
                if (i >= m) { i -= m; ++l; }
            }
        } else if (lane < nl) {
            for (int i = w; i < m; i += nw) {
                TW *pd = dst + b_lane + (int64_t)i * stride;
                const TW r = tile[lane * pitch + i];
                *pd = (p.vmode == 0) ? r : *pd + sg * r;
            }
        }
        __syncthreads();  // the tile is reused by the next panel
    }
}

}  // namespace mg
