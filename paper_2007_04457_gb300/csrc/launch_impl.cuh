// launch_impl.cuh -- definitions of the launchers declared in launch.cuh.
// Included only by the inst_*.cu translation units.
#pragma once

#include <algorithm>

#include "adjoint.cuh"
#include "interp.cuh"
#include "launch.cuh"
#include "multi.cuh"
#include "prolong.cuh"
#include "restrict.cuh"
#include "restrict_strip.cuh"
#include "small.cuh"
#include "sweep.cuh"
#include "solve.cuh"

namespace mg {

namespace detail {

struct RestrictEntry {
    void (*fn)(RestrictParams);
    int ty, tx;          // coarse rows / columns per tile (1D: coarse nodes per block)
    size_t smem;         // dynamic shared memory bytes
    int ipb;             // work items a block runs at once
};

template <typename T, typename TW, int ACT, int TY>
RestrictEntry restrict_entry()
{
    using G = RestrictGeom<T, ACT, TY>;
    return {k_restrict<T, TW, ACT, TY>, G::TY, kRestrictTX, sizeof(T) * (size_t)G::TOTAL, 1};
}

// Tile configuration 0 / 1 / 2 = 8 / 4 / 16 coarse rows; 3 = one warp per
// strip of 30 coarse columns (k_restrict_strip, 2D/3D only).  Both
// directions read a level array that holds coefficients on N_l \ N_{l-1}
// (the decomposition writes them before its restriction), so one kernel
// serves both.
template <typename T, typename TW, int ACT>
RestrictEntry restrict_pick_cfg(int cfg)
{
    if constexpr (ACT == ACT_1D) {
        return {k_restrict1d<T, TW>, 1, 256, 0, 1};
    } else {
        switch (cfg) {
        case 3:
            return {k_restrict_strip<T, TW, ACT == ACT_3D>, StripRows<T>::value, kStripCols, 0,
                    kStripThreads / 32};
        case 1: return restrict_entry<T, TW, ACT, 4>();
        case 2: return restrict_entry<T, TW, ACT, 16>();
        default: return restrict_entry<T, TW, ACT, 8>();
        }
    }
}

template <typename T, typename TW>
bool restrict_pick(int act, int cfg, RestrictEntry *e)
{
    if (cfg < 0 || cfg >= kRestrictConfigs) return false;
    if (cfg == 3 && act == ACT_1D) return false;
    switch (act) {
    case ACT_1D: *e = restrict_pick_cfg<T, TW, ACT_1D>(cfg); return true;
    case ACT_2D: *e = restrict_pick_cfg<T, TW, ACT_2D>(cfg); return true;
    case ACT_3D: *e = restrict_pick_cfg<T, TW, ACT_3D>(cfg); return true;
    default: return false;
    }
}

inline cudaError_t prepare(void (*fn)(RestrictParams), size_t smem, int *bps)
{
    if (smem > 0) {
        cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, kRestrictThreads, smem);
}

}  // namespace detail

template <typename T, typename TW>
cudaError_t restrict_shape(int act, int mode, int cfg, RestrictShape *out)
{
    (void)mode;
    detail::RestrictEntry e;
    if (!detail::restrict_pick<T, TW>(act, cfg, &e)) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t err = detail::prepare(e.fn, e.smem, &bps);
    if (err != cudaSuccess) return err;
    out->ty = e.ty;
    out->tx = e.tx;
    out->smem = e.smem;
    out->blocks_per_sm = bps;
    out->items_per_block = e.ipb;
    return cudaSuccess;
}

template <typename T, typename TW>
cudaError_t launch_restrict(int act, int mode, int cfg, const RestrictParams &p, int grid, cudaStream_t st)
{
    (void)mode;
    detail::RestrictEntry e;
    if (!detail::restrict_pick<T, TW>(act, cfg, &e)) return cudaErrorInvalidValue;
    { const cudaError_t le = launch_pdl(e.fn, dim3(grid), dim3(kRestrictThreads), e.smem, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

// k_solve_chunks: 16 nodes per warp and line up to 18 x 16 = 288 nodes, 32
// up to 576.
template <typename TW>
cudaError_t launch_solve_chunks(const SolveParams &p, int num_sms, cudaStream_t st)
{
    const int ch = (p.m <= 16 * kSolveChunkWarps) ? 16 : 32;
    const int nw = (p.m + ch - 1) / ch;
    const bool contig = (p.inner == 1);
    const size_t smem = solve_chunks_elems(p.m, nw, ch, contig) * sizeof(TW);
    void (*fn)(SolveParams);
    if (ch == 16) fn = contig ? k_solve_chunks<TW, 16, true> : k_solve_chunks<TW, 16, false>;
    else fn = contig ? k_solve_chunks<TW, 32, true> : k_solve_chunks<TW, 32, false>;
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 32 * nw, smem);
    if (err != cudaSuccess) return err;
    const int64_t panels = (p.nlines + 31) / 32;
    const int64_t grid = std::min<int64_t>(panels, (int64_t)std::max(1, bps) * num_sms);
    return launch_pdl(fn, dim3((unsigned)grid), dim3(32, nw), smem, st, p);
}

// k_solve_strided: chunks of CH = 17 nodes (preferred), 33 (4-byte elements
// only: 8-byte chunks of 33 do not fit the registers) or 9, nw = ceil(m / CH)
// <= 16 warps per panel of 32 lines; the kernel needs every chunk CH - 1 or
// CH nodes long, i.e. ceil(m / nw) = CH.  Returns 0 when no chunk length
// fits (the caller takes another kernel), else CH and *nw_out.
template <typename TW>
int solve_strided_shape(const SolveParams &p, int *nw_out)
{
    if (p.inner < 1 || p.nlines >= (int64_t(1) << 31) || p.inner >= (int64_t(1) << 31) ||
        (int64_t)p.m * p.stride >= (int64_t(1) << 31) || (size_t)4 * p.m * sizeof(TW) > 100 * 1024)
        return 0;
    static const int chs[3] = {17, 33, 9};
    for (int ch : chs) {
        if (sizeof(TW) == 8 && ch > 17) continue;
        const int nw = (p.m + ch - 1) / ch;
        if (nw >= 1 && nw <= kSolveStridedWarps && (p.m + nw - 1) / nw == ch) {
            *nw_out = nw;
            return ch;
        }
    }
    return 0;
}

// contiguous lines (inner = 1): k_solve_rowpanel, else k_solve_strided
template <typename TW>
cudaError_t launch_solve_strided(const SolveParams &p, int ch, int nw, int num_sms, cudaStream_t st)
{
    const bool rows = (p.inner == 1);
    void (*fn)(SolveParams);
    if (rows)
        fn = (ch == 17) ? k_solve_rowpanel<TW, 17> : (ch == 33) ? k_solve_rowpanel<TW, 33> : k_solve_rowpanel<TW, 9>;
    else
        fn = (ch == 17) ? k_solve_strided<TW, 17> : (ch == 33) ? k_solve_strided<TW, 33> : k_solve_strided<TW, 9>;
    const size_t smem = (rows ? solve_rowpanel_elems<TW>(p.m, nw) : solve_strided_elems<TW>(p.m, nw)) * sizeof(TW);
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 32 * nw, smem);
    if (err != cudaSuccess) return err;
    const int64_t panels = (p.nlines + 31) / 32;
    const int64_t grid = std::min<int64_t>(panels, (int64_t)std::max(1, bps) * num_sms);
    return launch_pdl(fn, dim3((unsigned)grid), dim3(32 * nw), smem, st, p);
}

// k_solve_lines: one thread per line, the factors of the line in shared memory.
template <typename TW>
cudaError_t launch_solve_lines(const SolveParams &p, int num_sms, cudaStream_t st)
{
    const size_t smem = (size_t)3 * p.m * sizeof(TW);
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(k_solve_lines<TW>),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_solve_lines<TW>, kSolveLineThreads, smem);
    if (err != cudaSuccess) return err;
    const int64_t blocks = (p.nlines + kSolveLineThreads - 1) / kSolveLineThreads;
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)std::max(1, bps) * num_sms);
    { const cudaError_t le = launch_pdl(k_solve_lines<TW>, dim3((unsigned)grid), dim3(kSolveLineThreads), smem, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

// nw_req = -1: k_solve_lines (one thread per line); nw_req = 0: FP64
// working arrays along the slowest dimension (or strided lines too long for
// the register chunks) k_solve_lines, else where a chunk length fits
// k_solve_strided along a strided dimension and k_solve_rowpanel along the
// contiguous one, else k_solve_chunks for lines up to 576 nodes; else (or nw_req > 0) the shared-memory panel kernel with
// nw_req warps (0: about 16 nodes per chunk).
template <typename TW>
cudaError_t launch_solve(const SolveParams &p_in, int nw_req, int num_sms, cudaStream_t st)
{
    SolveParams p = p_in;
    if (p.nlines <= 0) return cudaSuccess;
    const bool lines_fit = (size_t)3 * p.m * sizeof(TW) <= 100 * 1024;
    if (lines_fit && nw_req == -1) return launch_solve_lines<TW>(p, num_sms, st);
    if (nw_req < 0) nw_req = 0;
    if (nw_req == 0) {
        int snw = 0;
        const int sch = solve_strided_shape<TW>(p, &snw);
        // FP64 working arrays are bound by the FP64 units, where the chunked
        // kernels' second pass over every chunk costs: one thread per line
        // (the least arithmetic) for the slowest dimension (nlines <= inner)
        // when it has at least 128 lines per SM, and for strided lines too
        // long for the register chunks (measured: 513^3 FP64 z solve 0.67 ->
        // 0.45 ms per step, 1025^2 x 513 mixed step 16.5 -> 13.2 ms; with
        // 16.6K lines the chunks stay faster, with 33K the lines)
        const bool slowest = p.nlines <= p.inner && p.nlines >= (int64_t)kSolveLinesPerSm * num_sms;
        if (sizeof(TW) == 8 && lines_fit && p.inner > 1 && (slowest || sch == 0))
            return launch_solve_lines<TW>(p, num_sms, st);
        // contiguous lines: the two staged panels must fit beside the tables
        const bool fits = p.inner > 1 || solve_rowpanel_elems<TW>(p.m, snw) * sizeof(TW) <= 110 * 1024;
        if (sch > 0 && fits) return launch_solve_strided<TW>(p, sch, snw, num_sms, st);
    }
    if (nw_req == 0 && p.m <= 32 * kSolveChunkWarps && (int64_t)p.m * p.stride < (int64_t(1) << 31)) {
        const int ch = (p.m <= 16 * kSolveChunkWarps) ? 16 : 32;
        const int nw = (p.m + ch - 1) / ch;
        if (solve_chunks_elems(p.m, nw, ch, p.inner == 1) * sizeof(TW) <= 200 * 1024)
            return launch_solve_chunks<TW>(p, num_sms, st);
    }
    int nw = nw_req > 0 ? nw_req : std::min(32, std::max(1, (p.m + 15) / 16));
    nw = std::max(1, std::min(nw, std::min(32, p.m)));
    p.nw = nw;
    p.chunk = (p.m + nw - 1) / nw;
    constexpr size_t kCap = 200 * 1024;
    int lpb = 32;
    while (lpb > 1 && solve_panel_elems(p.m, lpb) * sizeof(TW) > kCap) lpb /= 2;
    const size_t smem = solve_panel_elems(p.m, lpb) * sizeof(TW);
    if (smem > kCap) return cudaErrorInvalidValue;
    p.lpb = lpb;
    const bool reg = (p.chunk <= 16) && (nw <= kSolveRegWarps);
    void (*fn)(SolveParams) = reg ? k_solve_panel<TW, 16> : k_solve_panel<TW, 0>;
    // set on every call, like the other launchers: the attribute belongs to
    // the current device, and a process may drive several
    const cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCap);
    if (err != cudaSuccess) return err;
    const int64_t panels = (p.nlines + lpb - 1) / lpb;
    { const cudaError_t le = launch_pdl(fn, dim3((unsigned)std::min<int64_t>(panels, 1 << 30)), dim3(32, nw), smem, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

namespace detail {

// Block of a multiple of 32 threads (<= 256) that splits n evenly into chunks.
inline void node_grid(int64_t nx, int64_t ny, int64_t nz, dim3 *grid, dim3 *block)
{
    const int64_t chunks = (nx + 255) / 256;
    int64_t bx = (nx + chunks - 1) / chunks;
    bx = (bx + 31) / 32 * 32;
    *block = dim3((unsigned)bx);
    *grid = dim3((unsigned)((nx + bx - 1) / bx), (unsigned)std::min<int64_t>(ny, 65535),
                 (unsigned)std::min<int64_t>(nz, 65535));
}

// Plane chunking of k_sweep: enough warp items for about 16 resident warps
// per SM twice over, chunks of an even number of fine planes.
inline int64_t sweep_rows(int act, size_t elem)
{
    (void)elem;
    return (act & 2) ? 8 : 1;
}

inline void sweep_chunks(PlaceParams &p, int act, int64_t R, int num_sms)
{
    const int64_t tiles = ((p.n2 + 31) / 32) * ((act & 2) ? (p.n1 + R - 1) / R : 1);
    if (!(act & 4)) {
        p.zchunk = 1;
        p.nzc = 1;
        return;
    }
    const int64_t want = (int64_t)num_sms * 32;
    const int64_t nz = std::max<int64_t>(1, std::min<int64_t>((want + tiles - 1) / tiles, (p.n0 - 1) / 2));
    int64_t zc = (p.n0 + nz - 1) / nz;
    zc += zc & 1;
    p.zchunk = std::max<int64_t>(2, zc);
    p.nzc = (p.n0 + p.zchunk - 1) / p.zchunk;
}

// k_sweep2 (recomposition, 4-byte 2D/3D levels): tiles of 64 columns.
template <typename T, typename TW>
cudaError_t launch_sweep2(int act, PlaceParams p, int num_sms, cudaStream_t st)
{
    constexpr int64_t R = 8;
    const int64_t tiles = ((p.m2 + 31) / 32) * ((p.n1 + R - 1) / R);
    if (!(act & 4)) {
        p.zchunk = 1;
        p.nzc = 1;
    } else {
        const int64_t want = (int64_t)num_sms * 32;
        const int64_t nz = std::max<int64_t>(1, std::min<int64_t>((want + tiles - 1) / tiles, (p.n0 - 1) / 2));
        int64_t zc = (p.n0 + nz - 1) / nz;
        zc += zc & 1;
        p.zchunk = std::max<int64_t>(2, zc);
        p.nzc = (p.n0 + p.zchunk - 1) / p.zchunk;
    }
    const int64_t items = tiles * p.nzc;
    const int64_t blocks = std::min<int64_t>((items + kSweepWarps - 1) / kSweepWarps, 1 << 30);
    if (act == ACT_3D) { const cudaError_t le = launch_pdl(k_sweep2<T, TW, ACT_3D>, dim3((unsigned)blocks), dim3(32 * kSweepWarps), 0, st, p); if (le != cudaSuccess) return le; }
    else { const cudaError_t le = launch_pdl(k_sweep2<T, TW, ACT_2D>, dim3((unsigned)blocks), dim3(32 * kSweepWarps), 0, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

template <typename T, typename TW, int MODE>
cudaError_t launch_sweep(int act, PlaceParams p, int num_sms, cudaStream_t st)
{
    if (MODE == MODE_REC && sizeof(T) == 4 && act != ACT_1D) return launch_sweep2<T, TW>(act, p, num_sms, st);
    const int64_t R = sweep_rows(act, sizeof(T));
    sweep_chunks(p, act, R, num_sms);
    const int64_t items = ((p.n2 + 31) / 32) * ((act & 2) ? (p.n1 + R - 1) / R : 1) * p.nzc;
    const int64_t blocks = std::min<int64_t>((items + kSweepWarps - 1) / kSweepWarps, 1 << 30);
    switch (act) {
    case ACT_1D: return launch_pdl(k_sweep<T, TW, ACT_1D, MODE>, dim3((unsigned)blocks), dim3(32 * kSweepWarps), 0, st, p);
    case ACT_2D: return launch_pdl(k_sweep<T, TW, ACT_2D, MODE>, dim3((unsigned)blocks), dim3(32 * kSweepWarps), 0, st, p);
    case ACT_3D: return launch_pdl(k_sweep<T, TW, ACT_3D, MODE>, dim3((unsigned)blocks), dim3(32 * kSweepWarps), 0, st, p);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace detail

template <typename T, typename TW>
cudaError_t launch_coef(int act, const PlaceParams &p, int num_sms, cudaStream_t st)
{
    return detail::launch_sweep<T, TW, MODE_DEC>(act, p, num_sms, st);
}

template <typename T, typename TW>
cudaError_t launch_scatter(int act, const PlaceParams &p, cudaStream_t st)
{
    const int64_t rows = p.m0 * p.m1;
    const int64_t blocks = std::min<int64_t>((rows + kScatterWarps - 1) / kScatterWarps, 1 << 20);
    const dim3 g((unsigned)blocks), b(32 * kScatterWarps);
    switch (act) {
    case ACT_1D: return launch_pdl(k_scatter<T, TW, ACT_1D>, g, b, 0, st, p);
    case ACT_2D: return launch_pdl(k_scatter<T, TW, ACT_2D>, g, b, 0, st, p);
    case ACT_3D: return launch_pdl(k_scatter<T, TW, ACT_3D>, g, b, 0, st, p);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_interp(int act, const PlaceParams &p, int num_sms, cudaStream_t st)
{
    return detail::launch_sweep<T, TW, MODE_REC>(act, p, num_sms, st);
}

#define MG_ACT_SWITCH(KERNEL, G, B, P)                                          \
    switch (act) {                                                             \
    case ACT_1D: return launch_pdl(KERNEL<T, TW, ACT_1D>, G, B, 0, st, P);     \
    case ACT_2D: return launch_pdl(KERNEL<T, TW, ACT_2D>, G, B, 0, st, P);     \
    case ACT_3D: return launch_pdl(KERNEL<T, TW, ACT_3D>, G, B, 0, st, P);     \
    default: return cudaErrorInvalidValue;                                     \
    }

template <typename T, typename TW>
cudaError_t launch_gather(int act, const PlaceParams &p, cudaStream_t st)
{
    dim3 g, b;
    detail::node_grid(p.m2, p.m1, p.m0, &g, &b);
    MG_ACT_SWITCH(k_gather, g, b, p)
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_adj_odd(int act, const AdjParams &p, cudaStream_t st)
{
    const size_t smem2 = (size_t)kAdj2Warps * 4 * p.m2 * sizeof(TW);
    if (act != ACT_1D && smem2 <= 96 * 1024) {
        void (*fn)(AdjParams) = (act == ACT_3D) ? k_adj_odd2<T, TW, ACT_3D> : k_adj_odd2<T, TW, ACT_2D>;
        cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (err != cudaSuccess) return err;
        const int64_t items = ((act == ACT_3D) ? (p.n0 + 1) / 2 : 1) * ((p.n1 + 1) / 2);
        const int64_t blocks = std::min<int64_t>((items + kAdj2Warps - 1) / kAdj2Warps, int64_t(1) << 30);
        { const cudaError_t le = launch_pdl(fn, dim3((unsigned)blocks), dim3(32 * kAdj2Warps), smem2, st, p); if (le != cudaSuccess) return le; }
        return cudaGetLastError();
    }
    dim3 g, b;
    detail::node_grid(p.n2, p.n1, p.n0, &g, &b);
    MG_ACT_SWITCH(k_adj_odd, g, b, p)
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_adj_even(int act, const AdjParams &p, cudaStream_t st)
{
    if (act != ACT_1D) {
        const int64_t items = p.m0 * p.m1;
        const int64_t blocks = std::min<int64_t>((items + kAdj2Warps - 1) / kAdj2Warps, int64_t(1) << 30);
        if (act == ACT_3D) { const cudaError_t le = launch_pdl(k_adj_even2<T, TW, ACT_3D>, dim3((unsigned)blocks), dim3(32 * kAdj2Warps), 0, st, p); if (le != cudaSuccess) return le; }
        else { const cudaError_t le = launch_pdl(k_adj_even2<T, TW, ACT_2D>, dim3((unsigned)blocks), dim3(32 * kAdj2Warps), 0, st, p); if (le != cudaSuccess) return le; }
        return cudaGetLastError();
    }
    dim3 g, b;
    detail::node_grid(p.m2, p.m1, p.m0, &g, &b);
    MG_ACT_SWITCH(k_adj_even, g, b, p)
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_small(int mode, const SmallParams &p, size_t smem, cudaStream_t st)
{
    void (*fn)(SmallParams) = (mode == MODE_DEC) ? k_small<T, TW, MODE_DEC> : k_small<T, TW, MODE_REC>;
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    { const cudaError_t le = launch_pdl(fn, dim3(1), dim3(kSmallThreads), smem, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_small_adj(int dir, const SmallParams &p, size_t smem, cudaStream_t st)
{
    void (*fn)(SmallParams) = (dir == 0) ? k_small_adj<T, TW, 0> : k_small_adj<T, TW, 1>;
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    { const cudaError_t le = launch_pdl(fn, dim3(1), dim3(kSmallThreads), smem, st, p); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

template <typename TX, typename TW>
cudaError_t multi_occupancy(int mode, size_t smem, int *blocks_per_sm)
{
    void (*fn)(MultiParams) = (mode == MODE_DEC) ? k_multi<TX, TW, MODE_DEC> : k_multi<TX, TW, MODE_REC>;
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kMultiThreads, smem);
}

template <typename TX, typename TW>
cudaError_t launch_multi(int mode, const MultiParams &p, int grid, size_t smem, cudaStream_t st)
{
    void (*fn)(MultiParams) = (mode == MODE_DEC) ? k_multi<TX, TW, MODE_DEC> : k_multi<TX, TW, MODE_REC>;
    // the limit is per function: plans with other shapes may have lowered it
    cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kMultiThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, p);
}

template <typename T, typename TW>
cudaError_t launch_prolong(const ProlongParams &p, int num_sms, cudaStream_t st)
{
    if (p.shift < 1 || p.n0 < 1 || p.n1 < 1 || p.n2 < 1) return cudaErrorInvalidValue;
    // one wave of resident blocks (the grid-stride loop covers the rest)
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prolong<T, TW>, kProlongThreads, 0);
    if (err != cudaSuccess) return err;
    per_sm = std::max(1, std::min(per_sm, kProlongBlocksPerSm));
    ProlongParams q = p;
    const int64_t rows = (int64_t)p.n0 * p.n1;
    const int64_t warps = (int64_t)num_sms * per_sm * (kProlongThreads / 32);
    // whole rows per work item when there are enough rows, else 256 nodes
    q.seg = (rows >= 4 * warps) ? (p.n2 + 31) / 32 * 32 : 256;
    const int64_t items = rows * ((p.n2 + q.seg - 1) / q.seg);
    if (items >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    const int64_t need = (items + kProlongThreads / 32 - 1) / (kProlongThreads / 32);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * per_sm));
    { const cudaError_t le = launch_pdl(k_prolong<T, TW>, dim3((unsigned)grid), dim3(kProlongThreads), 0, st, q); if (le != cudaSuccess) return le; }
    return cudaGetLastError();
}

#define MG_INSTANTIATE_LEVEL(T, TW)                                                              \
    template cudaError_t restrict_shape<T, TW>(int, int, int, RestrictShape *);                  \
    template cudaError_t launch_restrict<T, TW>(int, int, int, const RestrictParams &, int,     \
                                                cudaStream_t);                                   \
    template cudaError_t launch_coef<T, TW>(int, const PlaceParams &, int, cudaStream_t);       \
    template cudaError_t launch_scatter<T, TW>(int, const PlaceParams &, cudaStream_t);         \
    template cudaError_t launch_interp<T, TW>(int, const PlaceParams &, int, cudaStream_t);    \
    template cudaError_t launch_gather<T, TW>(int, const PlaceParams &, cudaStream_t);         \
    template cudaError_t launch_adj_odd<T, TW>(int, const AdjParams &, cudaStream_t);          \
    template cudaError_t launch_adj_even<T, TW>(int, const AdjParams &, cudaStream_t);          \
    template cudaError_t launch_small<T, TW>(int, const SmallParams &, size_t, cudaStream_t);    \
    template cudaError_t launch_small_adj<T, TW>(int, const SmallParams &, size_t, cudaStream_t); \
    template cudaError_t multi_occupancy<T, TW>(int, size_t, int *);                             \
    template cudaError_t launch_multi<T, TW>(int, const MultiParams &, int, size_t, cudaStream_t); \
    template cudaError_t launch_prolong<T, TW>(const ProlongParams &, int, cudaStream_t);

#define MG_INSTANTIATE_SOLVE(TW) \
    template cudaError_t launch_solve<TW>(const SolveParams &, int, int, cudaStream_t);

}  // namespace mg
