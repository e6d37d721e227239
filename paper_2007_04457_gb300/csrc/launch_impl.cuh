// launch_impl.cuh -- definitions of the launchers declared in launch.cuh.
// Included only by the inst_*.cu translation units.
#pragma once

#include "interp.cuh"
#include "launch.cuh"
#include "restrict.cuh"
#include "solve.cuh"

namespace mg {

namespace detail {

struct RestrictEntry {
    void (*fn)(RestrictParams);
    int ty, tx;
    size_t smem;
};

template <typename T, typename TW, int ACT, int MODE, int TY>
RestrictEntry restrict_entry()
{
    using G = RestrictGeom<T, ACT, MODE, TY>;
    return {k_restrict<T, TW, ACT, MODE, TY>, G::TY, kRestrictTX, sizeof(T) * (size_t)G::TOTAL};
}

template <typename T, typename TW, int ACT, int MODE>
RestrictEntry restrict_pick_cfg(int cfg)
{
    if constexpr (ACT == ACT_1D) {
        return {k_restrict1d<T, TW, MODE>, 1, 256, 0};
    } else {
        switch (cfg) {
        case 1: return restrict_entry<T, TW, ACT, MODE, 4>();
        case 2: return restrict_entry<T, TW, ACT, MODE, 16>();
        default: return restrict_entry<T, TW, ACT, MODE, 8>();
        }
    }
}

template <typename T, typename TW>
bool restrict_pick(int act, int mode, int cfg, RestrictEntry *e)
{
    if (cfg < 0 || cfg >= kRestrictConfigs) return false;
    const bool dec = (mode == MODE_DEC);
    switch (act) {
    case ACT_1D: *e = dec ? restrict_pick_cfg<T, TW, ACT_1D, MODE_DEC>(cfg) : restrict_pick_cfg<T, TW, ACT_1D, MODE_REC>(cfg); return true;
    case ACT_2D: *e = dec ? restrict_pick_cfg<T, TW, ACT_2D, MODE_DEC>(cfg) : restrict_pick_cfg<T, TW, ACT_2D, MODE_REC>(cfg); return true;
    case ACT_3D: *e = dec ? restrict_pick_cfg<T, TW, ACT_3D, MODE_DEC>(cfg) : restrict_pick_cfg<T, TW, ACT_3D, MODE_REC>(cfg); return true;
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
    detail::RestrictEntry e;
    if (!detail::restrict_pick<T, TW>(act, mode, cfg, &e)) return cudaErrorInvalidValue;
    int bps = 0;
    cudaError_t err = detail::prepare(e.fn, e.smem, &bps);
    if (err != cudaSuccess) return err;
    out->ty = e.ty;
    out->tx = e.tx;
    out->smem = e.smem;
    out->blocks_per_sm = bps;
    return cudaSuccess;
}

template <typename T, typename TW>
cudaError_t launch_restrict(int act, int mode, int cfg, const RestrictParams &p, int grid, cudaStream_t st)
{
    detail::RestrictEntry e;
    if (!detail::restrict_pick<T, TW>(act, mode, cfg, &e)) return cudaErrorInvalidValue;
    e.fn<<<grid, kRestrictThreads, e.smem, st>>>(p);
    return cudaGetLastError();
}

template <typename TW>
cudaError_t launch_solve(const SolveParams &p_in, bool contiguous, bool use_smem, cudaStream_t st)
{
    SolveParams p = p_in;
    if (p.nlines <= 0) return cudaSuccess;
    if (use_smem || p.m > kRegLine) {
        // shared-memory chunks: as many lines per block as fit in 200 KB
        const size_t carry = sizeof(TW) * 2 * 32 * 32;
        const size_t per_line = sizeof(TW) * (size_t)(p.m | 1);
        int lpb = 32;
        while (lpb > 1 && carry + per_line * lpb > 200 * 1024) lpb /= 2;
        if (carry + per_line * lpb > 200 * 1024) return cudaErrorInvalidValue;
        p.lpb = lpb;
        p.nw = 32;
        p.chunk = (p.m + 31) / 32;
        const size_t smem = carry + per_line * lpb;
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(k_solve_smem<TW>),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (err != cudaSuccess) return err;
            attr_set = true;
        }
        const unsigned grid = (unsigned)((p.nlines + lpb - 1) / lpb);
        k_solve_smem<TW><<<grid, dim3(32, 32), smem, st>>>(p);
        return cudaGetLastError();
    }
    const dim3 block(32, p.nw);
    const unsigned grid = (unsigned)((p.nlines + 31) / 32);
    const size_t smem = sizeof(TW) * (2 * 32 * 32 + 32 * (size_t)(p.m | 1));
    const bool staged = contiguous;
    void (*fn)(SolveParams) = nullptr;
    if (p.chunk != 16) return cudaErrorInvalidValue;
    fn = staged ? k_solve_contig<TW, 16> : k_solve_strided<TW, 16>;
    if (staged) {
        if (smem > 48 * 1024) {
            cudaError_t err = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   200 * 1024);
            if (err != cudaSuccess) return err;
        }
        fn<<<grid, block, smem, st>>>(p);
    } else {
        fn<<<grid, block, 0, st>>>(p);
    }
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_place(int act, int phase, const PlaceParams &p, int grid, cudaStream_t st)
{
    switch (act * 2 + phase) {
    case ACT_1D * 2 + 1: k_place<T, TW, ACT_1D, 1><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_2D * 2 + 0: k_place<T, TW, ACT_2D, 0><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_2D * 2 + 1: k_place<T, TW, ACT_2D, 1><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_3D * 2 + 0: k_place<T, TW, ACT_3D, 0><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_3D * 2 + 1: k_place<T, TW, ACT_3D, 1><<<grid, kRowThreads, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, typename TW>
cudaError_t launch_interp(int act, const PlaceParams &p, int grid, cudaStream_t st)
{
    switch (act) {
    case ACT_1D: k_interp<T, TW, ACT_1D><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_2D: k_interp<T, TW, ACT_2D><<<grid, kRowThreads, 0, st>>>(p); break;
    case ACT_3D: k_interp<T, TW, ACT_3D><<<grid, kRowThreads, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

#define MG_INSTANTIATE_LEVEL(T, TW)                                                              \
    template cudaError_t restrict_shape<T, TW>(int, int, int, RestrictShape *);                  \
    template cudaError_t launch_restrict<T, TW>(int, int, int, const RestrictParams &, int,     \
                                                cudaStream_t);                                   \
    template cudaError_t launch_place<T, TW>(int, int, const PlaceParams &, int, cudaStream_t); \
    template cudaError_t launch_interp<T, TW>(int, const PlaceParams &, int, cudaStream_t);

#define MG_INSTANTIATE_SOLVE(TW) \
    template cudaError_t launch_solve<TW>(const SolveParams &, bool, bool, cudaStream_t);

}  // namespace mg
