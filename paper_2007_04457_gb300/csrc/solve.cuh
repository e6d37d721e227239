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
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
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


// ---------------------------------------------------------------------------
// k_solve_chunks: lane = line (a block takes a panel of 32 lines), warp w =
// nodes [w CH, w CH + CH) of every line, held in registers.  Both sweeps are
// first-order linear recurrences, so each warp runs its chunk from a zero
// carry and corrects afterwards:
//   forward   y_i = y_i^loc + Pf_i c_w,  Pf_i = prod_{k=s..i} (-a_k)
//   backward  z_i = z_i^loc + Qb_i d_w,  Qb_i = prod_{k=i..e} (-q_k)
// where the carries c_w (y at the end of the chunk before) and d_w (z at the
// start of the chunk after) are composed from the other warps' chunk-end
// values through shared memory.  Pf and Qb depend only on the factors, so
// they are tabulated once per block.  For a non-contiguous dimension every
// node index of the panel is a row of 32 adjacent elements, loaded straight
// into registers; lines along the contiguous dimension form one contiguous
// block, staged through shared memory with 16-byte copies.
// ---------------------------------------------------------------------------

// Shared memory of k_solve_chunks, in elements of TW: factors and
// corrections (5 m), carries (2 x 32 nw), and the staging buffers: CONTIG two
// panels of 32 lines x m; otherwise two F chunks and one V chunk per thread.
inline size_t solve_chunks_elems(int m, int nw, int ch, bool contig)
{
    const size_t stage = contig ? 2 * (size_t)((32 * m + 3) & ~3) : 3 * (size_t)nw * ch * 32;
    return 5 * (size_t)m + 2 * 32 * (size_t)nw + stage + 4;
}

// at most 18 warps (chunks) per block
constexpr int kSolveChunkWarps = 18;

template <typename TW, int CH, bool CONTIG>
__global__ void __launch_bounds__(32 * kSolveChunkWarps) k_solve_chunks(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = p.m, nw = blockDim.y;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane, nthr = 32 * nw;
    TW *sfac = reinterpret_cast<TW *>(smem_raw);  // a, inv, q per node
    TW *Pf = sfac + 3 * m;
    TW *Qb = Pf + m;
    TW *ca = Qb + m;                              // forward chunk-end values [nw][32]
    TW *cb = ca + 32 * nw;                        // backward chunk-start values [nw][32]
    TW *stg = reinterpret_cast<TW *>((reinterpret_cast<uintptr_t>(cb + 32 * nw) + 15) & ~uintptr_t(15));
    // CONTIG: two panel buffers of tpitch elements; otherwise per thread two
    // F chunks and a V chunk, element j of thread (w, lane) at (w CH + j) 32 + lane
    const int tpitch = (32 * m + 3) & ~3;
    const int cpitch = nw * CH * 32;
    TW *vst = stg + 2 * cpitch;
    const TW *fac = static_cast<const TW *>(p.fac);
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *in = p.src ? static_cast<const TW *>(p.src) : F;
    const int s = w * CH;
    const int len = max(0, min(CH, m - s));
    const int64_t inner = p.inner;
    const int stride = (int)p.stride;  // a line spans m * stride < 2^31 elements (checked by the launcher)
    const int64_t npanels = (p.nlines + 31) / 32;

    for (int i = tid; i < 3 * m; i += nthr) sfac[i] = fac[i];
    __syncthreads();
    if (lane == 0) {
        TW pr = TW(1);
        for (int j = 0; j < len; ++j) {
            pr = -sfac[3 * (s + j)] * pr;
            Pf[s + j] = pr;
        }
        pr = TW(1);
        for (int j = len - 1; j >= 0; --j) {
            pr = -sfac[3 * (s + j) + 2] * pr;
            Qb[s + j] = pr;
        }
    }

    auto lines_of = [&](int64_t panel) { return (int)min64(32, p.nlines - panel * 32); };
    auto base_of = [&](int64_t panel) {
        const int64_t line = panel * 32 + min(lane, lines_of(panel) - 1);
        return line / inner * (inner * m) + line % inner;
    };
    // asynchronous staging of a panel into buffer b
    auto stage = [&](int64_t panel, int b) {
        if (panel >= npanels) return;
        if constexpr (CONTIG) {
            // the panel's lines are one contiguous block, 16-byte aligned
            const TW *src = in + panel * 32 * m;
            TW *dst = stg + b * tpitch;
            const int tot = lines_of(panel) * m;
            constexpr int E = 16 / sizeof(TW);
            const int nchunk = tot / E;
            for (int c = tid; c < nchunk; c += nthr) cp_async16(dst + c * E, src + c * E);
            for (int e = nchunk * E + tid; e < tot; e += nthr) cp_async_elem(dst + e, src + e, true);
        } else {
            // each thread copies its own chunk of its own line
            const bool lv = lane < lines_of(panel);
            const TW *src = in + base_of(panel) + (int64_t)s * stride;
            TW *dst = stg + b * cpitch + s * 32 + lane;
            for (int j = 0; j < len; ++j) cp_async_elem(dst + j * 32, lv ? src + j * stride : in, lv);
        }
    };

    int buf = 0;
    pdl_wait();  // the predecessor on the stream has finished with F and V
    stage(blockIdx.x, 0);
    cp_async_commit();
    __syncthreads();  // Pf, Qb ready

    for (int64_t panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
        const int nl = lines_of(panel);
        const bool lv = lane < nl;
        const int64_t base = CONTIG ? 0 : base_of(panel);
        // V of this panel (fused update), then the next panel, in flight
        // during the solve as two separate copy groups
        if (!CONTIG && p.vmode != 0) {
            const TW *src = V + base + (int64_t)s * stride;
            TW *dst = vst + s * 32 + lane;
            for (int j = 0; j < len; ++j) cp_async_elem(dst + j * 32, lv ? src + j * stride : V, lv);
        }
        cp_async_commit();
        stage(panel + gridDim.x, buf ^ 1);
        cp_async_commit();
        cp_async_wait<2>();  // this panel's staging is complete
        if constexpr (CONTIG) __syncthreads();
        TW y[CH];
        if constexpr (CONTIG) {
            const TW *t = stg + buf * tpitch;
#pragma unroll
            for (int j = 0; j < CH; ++j) y[j] = (j < len && lv) ? t[lane * m + s + j] : TW(0);
        } else {
            const TW *t = stg + buf * cpitch + s * 32 + lane;
#pragma unroll
            for (int j = 0; j < CH; ++j) y[j] = (j < len) ? t[j * 32] : TW(0);
        }
        // forward sweep
        TW t = TW(0);
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (j < len) {
                t = y[j] - sfac[3 * (s + j)] * t;
                y[j] = t;
            }
        ca[w * 32 + lane] = t;
        __syncthreads();
        TW c = TW(0);
        for (int k = 0; k < w; ++k) c = ca[k * 32 + lane] + Pf[min(k * CH + CH, m) - 1] * c;
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (j < len) y[j] += Pf[s + j] * c;
        // backward sweep
        t = TW(0);
#pragma unroll
        for (int j = CH - 1; j >= 0; --j)
            if (j < len) {
                t = sfac[3 * (s + j) + 1] * y[j] - sfac[3 * (s + j) + 2] * t;
                y[j] = t;
            }
        cb[w * 32 + lane] = t;
        __syncthreads();
        c = TW(0);
        for (int k = nw - 1; k > w; --k) c = cb[k * 32 + lane] + Qb[k * CH] * c;
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (j < len) y[j] += Qb[s + j] * c;
        // result: z into F, or V +- z
        const TW sg = (p.vmode == 2) ? TW(-1) : TW(1);
        if constexpr (CONTIG) {
            TW *t2 = stg + buf * tpitch;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (j < len && lv) t2[lane * m + s + j] = y[j];
            __syncthreads();
            TW *dst = ((p.vmode == 0) ? F : V) + panel * 32 * m;
            for (int e = tid; e < nl * m; e += nthr) dst[e] = (p.vmode == 0) ? t2[e] : dst[e] + sg * t2[e];
        } else {
            cp_async_wait<1>();  // the V chunk
            TW *dst = ((p.vmode == 0) ? F : V) + base + (int64_t)s * stride;
            const TW *vv = vst + s * 32 + lane;
            if (lv) {
#pragma unroll
                for (int j = 0; j < CH; ++j)
                    if (j < len) dst[j * stride] = (p.vmode == 0) ? y[j] : vv[j * 32] + sg * y[j];
            }
        }
        buf ^= 1;
        __syncthreads();  // carries and buffers are reused by the next panel
    }
    cp_async_wait<0>();
}

// k_solve_strided: lines along a dimension that is not the contiguous one.
// A block takes panels of 32 consecutive lines (lane = line: every load and
// store of a warp touches 32 neighbouring elements), its nw warps a chunk of
// every line each (chunk w = nodes [w m / nw, (w + 1) m / nw), CH - 1 or CH
// of them), held in registers together with the V values it updates.  Per
// sweep a warp runs its chunk's recurrence from a zero carry, publishes the
// chunk-end value, composes the carries of the chunks before it (each chunk
// is the affine map y_out = T + P y_in, P the product of its -a_i, or of its
// -q_i backward, tabulated per warp) and re-runs the chunk from its true
// carry.  The factors of a node are packed (a, inv, q) in shared memory and
// read with one vector load where they are used.  DRAM traffic: F read once,
// written once (or V read and written once).
template <typename TW>
inline size_t solve_strided_elems(int m, int nw)
{
    return 4 * (size_t)m + 2 * (size_t)nw + 2 * 32 * (size_t)nw;
}

constexpr int kSolveStridedWarps = 16;

// Registers sized for two blocks per SM where the chunk and its V values fit
// them (4-byte elements, CH <= 17), else one.
template <typename TW, int CH>
struct StridedMinBlocks {
    static constexpr int value = (sizeof(TW) == 4 && CH <= 17) ? 2 : 1;
};

// (a, inv, q) of one node from its packed shared-memory entry, loaded where
// it is used (an asm load: the compiler keeps no copy in registers)
__device__ __forceinline__ void solve_fac(const float *e, float &a, float &inv, float &q)
{
    float pad;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a), "=f"(inv), "=f"(q), "=f"(pad)
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(e))));
}

__device__ __forceinline__ void solve_fac(const double *e, double &a, double &inv, double &q)
{
    double pad;
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(e));
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(inv) : "r"(s));
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(q), "=d"(pad) : "r"(s + 16));
}

// Shared memory of the chunked solves: the packed factors (4 m), the chunk
// products Pw, Qw (nw each) and the carries ca, cb (32 nw each), in TW.
template <typename TW>
struct ChunkSmem {
    TW *sfac, *Pw, *Qw, *ca, *cb;
};

// Packs the factors of the line's nodes as (a, inv, q, 0) and tabulates each
// chunk's products of its -a_i and -q_i; chunk w = nodes [w m / nw,
// (w + 1) m / nw).  Reads only the plan's factor table.
template <typename TW>
__device__ __forceinline__ ChunkSmem<TW> chunk_setup(unsigned char *smem_raw, const TW *fac, int m, int w, int nw,
                                                     int lane)
{
    ChunkSmem<TW> c;
    c.sfac = reinterpret_cast<TW *>(smem_raw);
    c.Pw = c.sfac + 4 * m;
    c.Qw = c.Pw + nw;
    c.ca = c.Qw + nw;
    c.cb = c.ca + 32 * nw;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        c.sfac[4 * i] = fac[3 * i];
        c.sfac[4 * i + 1] = fac[3 * i + 1];
        c.sfac[4 * i + 2] = fac[3 * i + 2];
        c.sfac[4 * i + 3] = TW(0);
    }
    __syncthreads();
    const int s = (w * m) / nw, len = ((w + 1) * m) / nw - s;
    if (lane == 0) {
        TW pa = TW(1), pq = TW(1);
        for (int j = 0; j < len; ++j) {
            pa = -c.sfac[4 * (s + j)] * pa;
            pq = -c.sfac[4 * (s + j) + 2] * pq;
        }
        c.Pw[w] = pa;
        c.Qw[w] = pq;
    }
    __syncthreads();
    return c;
}

// M_{l-1} z = f on chunk w of the 32 lines of a panel (lane = line): y holds
// the chunk's right-hand sides (CH - 1 or CH of them: the last only when
// `full`); on return it holds z.  Per sweep the chunk runs from a zero carry,
// publishes its end value, composes the carries of the chunks before it and
// re-runs from its true carry.  Two block barriers; the caller puts one more
// between panels (the carries are reused).
template <typename TW, int CH>
__device__ __forceinline__ void chunk_solve_panel(TW (&y)[CH], const ChunkSmem<TW> &c, const TW *sf, bool full, int w,
                                                  int nw, int lane)
{
    TW a, inv, q;
    // forward y_i = f_i - a_i y_{i-1}: chunk-end value from a zero carry
    TW t = TW(0);
#pragma unroll
    for (int j = 0; j < CH; ++j)
        if (j < CH - 1 || full) {
            solve_fac(sf + 4 * j, a, inv, q);
            t = y[j] - a * t;
        }
    c.ca[w * 32 + lane] = t;
    __syncthreads();
    TW cr = TW(0);
    for (int k = 0; k < w; ++k) cr = c.ca[k * 32 + lane] + c.Pw[k] * cr;
    t = cr;
#pragma unroll
    for (int j = 0; j < CH; ++j)
        if (j < CH - 1 || full) {
            solve_fac(sf + 4 * j, a, inv, q);
            t = y[j] - a * t;
            y[j] = t;
        }
    // backward z_i = inv_i y_i - q_i z_{i+1}: chunk-start value from a zero carry
    t = TW(0);
#pragma unroll
    for (int j = CH - 1; j >= 0; --j)
        if (j < CH - 1 || full) {
            solve_fac(sf + 4 * j, a, inv, q);
            t = inv * y[j] - q * t;
        }
    c.cb[w * 32 + lane] = t;
    __syncthreads();
    cr = TW(0);
    for (int k = nw - 1; k > w; --k) cr = c.cb[k * 32 + lane] + c.Qw[k] * cr;
    t = cr;
#pragma unroll
    for (int j = CH - 1; j >= 0; --j)
        if (j < CH - 1 || full) {
            solve_fac(sf + 4 * j, a, inv, q);
            t = inv * y[j] - q * t;
            y[j] = t;
        }
}

template <typename TW, int CH>
__global__ void __launch_bounds__(32 * kSolveStridedWarps, StridedMinBlocks<TW, CH>::value) k_solve_strided(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = p.m;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const ChunkSmem<TW> cs = chunk_setup<TW>(smem_raw, static_cast<const TW *>(p.fac), m, w, nw, lane);
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *in = p.src ? static_cast<const TW *>(p.src) : F;
    const int s = (w * m) / nw, len = ((w + 1) * m) / nw - s;  // len is CH - 1 or CH
    const TW *sf = cs.sfac + 4 * s;
    const bool full = (len == CH);  // the chunk's last register holds a node
    pdl_wait();  // the predecessor on the stream has finished with F and V
    // line -> first element: lines are (outer, inner) pairs, inner fastest;
    // 32-bit arithmetic (the launcher checks that every index fits)
    const unsigned inner = (unsigned)p.inner, nlines = (unsigned)p.nlines;
    const int stride = (int)p.stride;
    const unsigned npanels = (nlines + 31) / 32;
    const TW sg = (p.vmode == 2) ? TW(-1) : TW(1);
    for (unsigned panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
        const unsigned line = panel * 32 + lane;
        const bool lv = line < nlines;
        const unsigned ln = lv ? line : nlines - 1;  // lanes past the end read the last line, store nothing
        const unsigned outer = (nlines <= inner) ? 0u : ln / inner;
        const int64_t base = (int64_t)outer * inner * m + (ln - outer * inner) + (int64_t)s * stride;
        const TW *fin = in + base;
        TW y[CH], vv[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) y[j] = (j < CH - 1 || full) ? fin[j * stride] : TW(0);
        if (p.vmode != 0) {
            const TW *vin = V + base;
#pragma unroll
            for (int j = 0; j < CH; ++j) vv[j] = (j < CH - 1 || full) ? vin[j * stride] : TW(0);
        }
        chunk_solve_panel<TW, CH>(y, cs, sf, full, w, nw, lane);
        // z into F, or V +- z
        if (lv) {
            TW *dst = ((p.vmode == 0) ? F : V) + base;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (j < CH - 1 || full) dst[j * stride] = (p.vmode == 0) ? y[j] : vv[j] + sg * y[j];
        }
        __syncthreads();  // the carries are reused by the next panel
    }
}

// k_solve_rowpanel: lines along the contiguous dimension.  A panel of 32
// consecutive lines is one contiguous, 16-byte aligned block of 32 m
// elements, staged with 16-byte cp.async copies into one of two buffers
// while the block solves the panel in the other (pitch m, odd, so that the
// lanes of a warp, one line each, read different banks); the chunked solve
// is the one of k_solve_strided; z goes back into the buffer and out with
// coalesced stores (z into F, or V +- z).
template <typename TW>
inline size_t solve_rowpanel_elems(int m, int nw)
{
    return solve_strided_elems<TW>(m, nw) + 4 + 2 * (size_t)((32 * m + 3) & ~3);
}

template <typename TW, int CH>
__global__ void __launch_bounds__(32 * kSolveStridedWarps, StridedMinBlocks<TW, CH>::value) k_solve_rowpanel(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = p.m;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const ChunkSmem<TW> cs = chunk_setup<TW>(smem_raw, static_cast<const TW *>(p.fac), m, w, nw, lane);
    TW *stg = reinterpret_cast<TW *>((reinterpret_cast<uintptr_t>(cs.cb + 32 * nw) + 15) & ~uintptr_t(15));
    const int tpitch = (32 * m + 3) & ~3;
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *in = p.src ? static_cast<const TW *>(p.src) : F;
    const int s = (w * m) / nw, len = ((w + 1) * m) / nw - s;  // len is CH - 1 or CH
    const TW *sf = cs.sfac + 4 * s;
    const bool full = (len == CH);
    const int64_t nlines = p.nlines, npanels = (nlines + 31) / 32;
    const TW sg = (p.vmode == 2) ? TW(-1) : TW(1);
    auto lines_of = [&](int64_t panel) { return (int)min64(32, nlines - panel * 32); };
    auto stage = [&](int64_t panel, int b) {
        if (panel >= npanels) return;
        const TW *src = in + panel * 32 * m;
        TW *dst = stg + b * tpitch;
        const int tot = lines_of(panel) * m;
        constexpr int E = 16 / sizeof(TW);
        const int nchunk = tot / E;
        for (int c = tid; c < nchunk; c += nthr) cp_async16(dst + c * E, src + c * E);
        for (int e = nchunk * E + tid; e < tot; e += nthr) cp_async_elem(dst + e, src + e, true);
    };
    pdl_wait();  // the predecessor on the stream has finished with F and V
    int buf = 0;
    stage(blockIdx.x, 0);
    cp_async_commit();
    for (int64_t panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
        stage(panel + gridDim.x, buf ^ 1);  // the next panel, in flight during this one
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int nl = lines_of(panel);
        TW *t = stg + buf * tpitch;
        const TW *row = t + min(lane, nl - 1) * m + s;  // lanes past the end solve a copy of the last line
        TW y[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) y[j] = (j < CH - 1 || full) ? row[j] : TW(0);
        chunk_solve_panel<TW, CH>(y, cs, sf, full, w, nw, lane);
        if (lane < nl) {
            TW *rw = t + lane * m + s;
#pragma unroll
            for (int j = 0; j < CH; ++j)
                if (j < CH - 1 || full) rw[j] = y[j];
        }
        __syncthreads();
        const int64_t g0 = panel * 32 * (int64_t)m;
        const int tot = nl * m;
        if (p.vmode == 0) {
            for (int e = tid; e < tot; e += nthr) F[g0 + e] = t[e];
        } else {
            for (int e = tid; e < tot; e += nthr) V[g0 + e] = V[g0 + e] + sg * t[e];
        }
        buf ^= 1;
        __syncthreads();  // the buffer, the carries: reused by the next panel
    }
    cp_async_wait<0>();
}

// One thread per line: the Thomas recurrences of the tabulated LU factors
// (forward y_i = f_i - a_i y_{i-1}, backward z_i = inv_i y_i - q_i z_{i+1}),
// U nodes at a time with the next U prefetched into registers before the
// current ones are stored, so a thread always has loads in flight.  Threads
// of a warp take consecutive lines: along a strided dimension their loads
// are coalesced, along the contiguous one each load instruction touches one
// 32-byte sector per lane that the next loads of the thread hit in L1.  The
// factors sit in shared memory as (a, inv, q) per node, read by every lane
// of the warp at the same address.  vmode as in SolveParams; the forward
// pass reads src when given and writes y into F, the backward pass writes z
// into F or V +- z into V.
constexpr int kSolveLineThreads = 256;
constexpr int kSolveLinesPerSm = 128;  // lines per SM from which one thread per line pays (FP64)

template <typename TW>
struct LineUnroll {
    static constexpr int value = sizeof(TW) == 4 ? 8 : 4;
};

template <typename TW>
__global__ void __launch_bounds__(kSolveLineThreads) k_solve_lines(SolveParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr int U = LineUnroll<TW>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *tab = reinterpret_cast<TW *>(smem_raw);
    const int m = p.m;
    const TW *fac = static_cast<const TW *>(p.fac);
    for (int e = threadIdx.x; e < 3 * m; e += blockDim.x) tab[e] = fac[e];
    __syncthreads();
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const TW *src = p.src ? static_cast<const TW *>(p.src) : F;
    const int64_t inner = p.inner, stride = p.stride;
    const int nch = (m + U - 1) / U;
    const TW sg = (p.vmode == 2) ? TW(-1) : TW(1);
    for (int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; line < p.nlines;
         line += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = (line / inner) * (inner * m) + line % inner;
        const TW *s_in = src + base;
        TW *f = F + base;
        // forward: y into F
        TW cur[U], nxt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = (u < m) ? s_in[(int64_t)u * stride] : TW(0);
        TW t = TW(0);
        for (int c = 0; c < nch; ++c) {
            const int k0 = c * U;
            if (c + 1 < nch) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    nxt[u] = (k0 + U + u < m) ? s_in[(int64_t)(k0 + U + u) * stride] : TW(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k0 + u < m) {
                    t = cur[u] - tab[3 * (k0 + u)] * t;
                    f[(int64_t)(k0 + u) * stride] = t;
                }
#pragma unroll
            for (int u = 0; u < U; ++u) cur[u] = nxt[u];
        }
        // backward: z into F, or V +- z
        TW *dst = (p.vmode == 0) ? f : V + base;
        TW vc[U], vn[U];
        {
            const int k0 = (nch - 1) * U;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cur[u] = (k0 + u < m) ? f[(int64_t)(k0 + u) * stride] : TW(0);
                vc[u] = (p.vmode != 0 && k0 + u < m) ? dst[(int64_t)(k0 + u) * stride] : TW(0);
            }
        }
        t = TW(0);
        for (int c = nch - 1; c >= 0; --c) {
            const int k0 = c * U;
            if (c > 0) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    nxt[u] = f[(int64_t)(k0 - U + u) * stride];
                    vn[u] = (p.vmode != 0) ? dst[(int64_t)(k0 - U + u) * stride] : TW(0);
                }
            }
#pragma unroll
            for (int u = U - 1; u >= 0; --u)
                if (k0 + u < m) {
                    t = tab[3 * (k0 + u) + 1] * cur[u] - tab[3 * (k0 + u) + 2] * t;
                    dst[(int64_t)(k0 + u) * stride] = (p.vmode == 0) ? t : vc[u] + sg * t;
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cur[u] = nxt[u];
                vc[u] = vn[u];
            }
        }
    }
}

}  // namespace mg
