// solve.cuh -- batched tridiagonal solves M_{l-1} z = f along one dimension
// of a compact coarse array (Section III-A-3: the correction solver, one
// Thomas solve per line).
//
// M_{l-1} is the same for every line of a dimension, so its LU factors are
// tabulated once per (level, dimension): forward y_i = f_i - a_i y_{i-1},
// backward z_i = inv_i y_i - q_i z_{i+1}.  Both sweeps are first-order linear
// recurrences; a line is split into `nw` chunks (one warp each, one lane per
// line), every chunk runs its recurrence from a zero carry while accumulating
// the product of its multipliers, the chunk carries are composed through
// shared memory, and each chunk re-runs with its true carry.  The chunk stays
// in registers, so every element is read and written once per sweep.
//
// k_solve_strided: lines along a non-contiguous dimension; the 32 lanes of a
//   warp take 32 consecutive lines, whose elements are adjacent in memory
//   (coalesced).
// k_solve_contig:  lines along the contiguous dimension; 32 lines are staged
//   through shared memory (coalesced in and out) and solved lane-per-line
//   from there.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

template <typename TW, int CH>
__device__ __forceinline__ void chunk_solve(TW (&r)[CH], const TW *__restrict__ fac, int s, int len, int w,
                                            int nw, TW *carry_a, TW *carry_b, int lane)
{
    // forward: local run from zero carry, product of (-a_i)
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
    // backward: z_i = inv_i y_i - q_i z_{i+1}, local run from zero carry
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
}

template <typename TW, int CH>
__global__ void __launch_bounds__(576) k_solve_strided(SolveParams p)
{
    __shared__ TW carry_a[32 * 32];
    __shared__ TW carry_b[32 * 32];
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *fac = static_cast<const TW *>(p.fac);
    const int lane = threadIdx.x, w = threadIdx.y;
    const int64_t line = (int64_t)blockIdx.x * 32 + lane;
    const bool active = line < p.nlines;
    const int64_t lc = active ? line : 0;
    const int64_t base = (lc / p.inner) * (p.inner * p.m) + (lc % p.inner);
    const int s = w * p.chunk;
    const int len = active ? max(0, min(p.chunk, p.m - s)) : 0;
    const int flen = max(0, min(p.chunk, p.m - s));  // same for all lanes: keeps fac reads uniform

    const int st = (int)p.stride;  // < 2^31 for every supported shape
    TW r[CH];
    {
        const TW *q = F + base + (int64_t)s * st;
#pragma unroll
        for (int j = 0; j < CH; ++j) r[j] = (j < len) ? q[j * st] : TW(0);
    }
    chunk_solve<TW, CH>(r, fac, s, flen, w, p.nw, carry_a, carry_b, lane);
    if (p.vmode == 0) {
        TW *q = F + base + (int64_t)s * st;
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (j < len) q[j * st] = r[j];
    } else {
        const TW sg = (p.vmode == 1) ? TW(1) : TW(-1);
        TW *q = V + base + (int64_t)s * st;
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (j < len) q[j * st] = q[j * st] + sg * r[j];
    }
}

template <typename TW, int CH>
__global__ void __launch_bounds__(576) k_solve_contig(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *carry_a = reinterpret_cast<TW *>(smem_raw);
    TW *carry_b = carry_a + 32 * 32;
    TW *tile = carry_b + 32 * 32;  // 32 lines, pitch m | 1
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *fac = static_cast<const TW *>(p.fac);
    const int lane = threadIdx.x, w = threadIdx.y;
    const int tid = w * 32 + lane, nthr = 32 * p.nw;
    const int m = p.m, pitch = m | 1;
    const int64_t line0 = (int64_t)blockIdx.x * 32;
    const int nl = (int)min64(32, p.nlines - line0);
    const TW *src = F + line0 * m;

    {
        int l = tid / m, i = tid - (tid / m) * m;
        for (int e = tid; e < nl * m; e += nthr) {
            tile[l * pitch + i] = src[e];
            i += nthr;
            while (i >= m) { i -= m; ++l; }
        }
    }
    __syncthreads();
    const int s = w * p.chunk;
    const int len = max(0, min(p.chunk, m - s));
    TW r[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) r[j] = (j < len && lane < nl) ? tile[lane * pitch + s + j] : TW(0);
    chunk_solve<TW, CH>(r, fac, s, len, w, p.nw, carry_a, carry_b, lane);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CH; ++j)
        if (j < len && lane < nl) tile[lane * pitch + s + j] = r[j];
    __syncthreads();
    if (p.vmode == 0) {
        TW *dst = F + line0 * m;
        int l = tid / m, i = tid - (tid / m) * m;
        for (int e = tid; e < nl * m; e += nthr) {
            dst[e] = tile[l * pitch + i];
            i += nthr;
            while (i >= m) { i -= m; ++l; }
        }
    } else {
        const TW sg = (p.vmode == 1) ? TW(1) : TW(-1);
        TW *dst = V + line0 * m;
        int l = tid / m, i = tid - (tid / m) * m;
        for (int e = tid; e < nl * m; e += nthr) {
            dst[e] = dst[e] + sg * tile[l * pitch + i];
            i += nthr;
            while (i >= m) { i -= m; ++l; }
        }
    }
}

// Long lines (more than 18 chunks of 16): the chunks stay in shared memory
// instead of registers.  `p.lpb` lines per block (<= 32, lanes >= lpb idle),
// 32 warps, chunk length p.chunk = ceil(m / 32).
template <typename TW>
__device__ __forceinline__ void chunk_solve_smem(TW *row, const TW *__restrict__ fac, int s, int len, int w,
                                                 int nw, TW *carry_a, TW *carry_b, int lane)
{
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

template <typename TW>
__global__ void __launch_bounds__(1024) k_solve_smem(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *carry_a = reinterpret_cast<TW *>(smem_raw);
    TW *carry_b = carry_a + 32 * 32;
    TW *tile = carry_b + 32 * 32;  // p.lpb lines, pitch m | 1
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *fac = static_cast<const TW *>(p.fac);
    const int lane = threadIdx.x, w = threadIdx.y;
    const int m = p.m, pitch = m | 1, lpb = p.lpb;
    const int64_t line0 = (int64_t)blockIdx.x * lpb;
    const int nl = (int)min64(lpb, p.nlines - line0);
    const int s = w * p.chunk;
    const int len = max(0, min(p.chunk, m - s));
    // element i of line l lives at base(l) + i * stride
    auto base = [&](int64_t line) { return (line / p.inner) * (p.inner * m) + (line % p.inner); };
    // load: warp w brings chunk w of every line of the block
    if (lane < nl) {
        const int64_t b = base(line0 + lane);
        for (int j = 0; j < len; ++j) tile[lane * pitch + s + j] = F[b + (int64_t)(s + j) * p.stride];
    }
    __syncthreads();
    chunk_solve_smem<TW>(tile + lane * pitch, fac, s, len, w, p.nw, carry_a, carry_b, lane);
    __syncthreads();
    if (lane < nl) {
        const int64_t b = base(line0 + lane);
        if (p.vmode == 0) {
            for (int j = 0; j < len; ++j) F[b + (int64_t)(s + j) * p.stride] = tile[lane * pitch + s + j];
        } else {
            const TW sg = (p.vmode == 1) ? TW(1) : TW(-1);
            for (int j = 0; j < len; ++j) {
                TW *pv = V + b + (int64_t)(s + j) * p.stride;
                *pv = *pv + sg * tile[lane * pitch + s + j];
            }
        }
    }
}

}  // namespace mg
