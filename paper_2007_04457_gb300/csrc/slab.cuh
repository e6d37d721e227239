// slab.cuh -- load vector and coarse gather of a 3D level from whole-row
// slabs that bulk asynchronous copies stage in shared memory.
//
// Computes, like k_restrict and k_restrict_strip (Section II-A Eq. 2; the
// mass-transfer stencil K = P^T M_l of Section III-A-2 along each dimension)
//   F = (K_0 (x) K_1 (x) K_2) C,  C = A on N_l \ N_{l-1}, 0 on N_{l-1}
//   V = A restricted to N_{l-1}
// for 3D level arrays of 4-byte elements whose rows have n2 = 64 k + 1
// nodes (m2 - 1 = (n2 - 1) / 2 threads per block, k = 1 .. 16).
//
// A block item is a band of TY coarse rows [Y0, Y0 + TY) over the whole row
// width and a chunk of coarse planes [Zs, Ze).  The fine rows 2 Y0 - 2 ..
// 2 Y0 + 2 TY of a fine plane, which feed the band, are one contiguous range
// of the array: thread 0 copies it into a ring slot with one cp.async.bulk
// (its 16-byte aligned cover), counted on the slot's mbarrier, up to NS - 1
// planes ahead of their use and across item boundaries (the block knows its
// whole item sequence).  Thread t owns coarse column t: per fine row it reads
// fine columns 2t - 2 .. 2t + 2 from the slot as three 8-byte pairs
// (conflict-free across a warp; every row starts at its own offset since n2
// is odd, the two pair alignments are compiled separately), applies the
// dim-2 stencil and accumulates the dim-1 stencil into TY register rows; the
// dim-0 stencil goes into rolling register accumulators over the planes of
// the chunk.  The last warp also computes the final column m2 - 1 (lane j
// its coarse row Y0 + j).  Optionally (XS) each finished coarse plane's rows
// are solved along dim 2 before they are stored.
//
// A band that would pass the last coarse row is shifted back to end there;
// its rows that the previous band owns are computed but not stored.  Every
// wait for a copy is bounded: when one runs out the block records bit 0 in
// *status, waits (bounded again) for the copies it has issued, and returns.
#pragma once

#include "common.cuh"
#include "params.h"
#include "rowchunk.cuh"  // rc_xsolve: a row's tridiagonal solve by one warp

namespace mg {

// ---- mbarrier and bulk-copy primitives (sm_90 and later)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised barriers visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// the arrival of the copy's issuer, announcing `bytes` of transfer
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (both addresses and the size 16-byte multiples)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// one arrival (release: the caller's earlier shared-memory accesses are
// ordered before it)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `parity` to complete; false when `limit_ns` passes
// first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ---- the kernel

template <int N>
struct SlabIC {
    static constexpr int value = N;
};

// f(SlabIC<I>{}) for I = B .. E - 1, unrolled at compile time
template <int B, int E, typename Fn>
__device__ __forceinline__ void slab_for(Fn &&f)
{
    if constexpr (B < E) {
        f(SlabIC<B>{});
        slab_for<B + 1, E>(f);
    }
}

constexpr int kSlabBarBytes = 256;  // ring barriers (full, then empty), ahead of the slots

template <int TY>
struct SlabGeom {
    static constexpr int NR = 2 * TY + 3;  // fine rows feeding TY coarse rows
};

// Bytes of a ring slot for rows of n2 4-byte nodes: NR rows plus the
// 16-byte rounding at both ends.
template <int TY>
__host__ __device__ inline int slab_slot_bytes(int n2)
{
    return ((SlabGeom<TY>::NR * n2 * 4 + 32) + 15) / 16 * 16;
}

// Bytes after the ring for the solve along dim 2 (XS): two buffers of TY
// rows of m2 (+1) coarse values and the factor table of a row (3 (m2 - 1)
// values, the final node's apart), in TW.
template <int TY>
__host__ __device__ inline int slab_xs_bytes(int n2, int tw_bytes)
{
    const int m2 = (n2 - 1) / 2 + 1;
    return ((2 * TY * (m2 + 1) + 3 * (m2 - 1)) * tw_bytes + 15) / 16 * 16;
}

// Item geometry: band b = item % nb, chunk c = item / nb.
struct SlabItem {
    int yown, Y0, Zs, Ze, zlo, zhi;
};

template <int TY>
__device__ __forceinline__ SlabItem slab_item(const SlabParams &p, int item)
{
    SlabItem it;
    const int b = item % p.nb, c = item / p.nb;
    it.yown = TY * b;
    it.Y0 = min(it.yown, p.m1 - TY);
    it.Zs = c * p.zchunk;
    it.Ze = (c == p.nzc - 1) ? p.m0 : it.Zs + p.zchunk;
    // fine planes 2 Zs - 2 (their taps reach coarse plane Zs) .. 2 Ze (tap 4
    // of coarse plane Ze - 1); the last chunk ends at the grid's last plane
    it.zlo = (it.Zs > 0) ? 2 * it.Zs - 2 : 0;
    it.zhi = 2 * min(it.Ze, p.m0 - 1);
    return it;
}

// Element offset (in 4-byte nodes, mod 4) of fine row 2 Y0 - 2 of plane z:
// the ring slot holds the 16-byte aligned cover of that row onward.
__device__ __forceinline__ int slab_s0(const float *A, int64_t plane, int n2, int z, int Y0)
{
    const int64_t e = (int64_t)(reinterpret_cast<uintptr_t>(A) >> 2) + (int64_t)z * plane + (int64_t)(2 * Y0 - 2) * n2;
    return (int)(e & 3);
}

// Issue the copy of fine plane z, rows 2 Y0 - 2 .. 2 Y0 + 2 TY (those
// inside the grid), into `slot`, counted on `bar`.  `extra` bytes are
// announced on top (a test hook: such a phase never completes).
template <int TY>
__device__ __forceinline__ void slab_issue(const float *A, int64_t plane, int n1, int n2, int z, int Y0,
                                           unsigned char *slot, uint64_t *bar, unsigned extra)
{
    const int ylo = max(2 * Y0 - 2, 0), yhi = min(2 * Y0 + 2 * TY, n1 - 1);
    const intptr_t base = reinterpret_cast<intptr_t>(A) + (intptr_t)z * plane * 4;
    const intptr_t vo = (base + (intptr_t)(2 * Y0 - 2) * n2 * 4) & ~(intptr_t)15;  // slot origin
    const intptr_t lo = (base + (intptr_t)ylo * n2 * 4) & ~(intptr_t)15;
    const intptr_t hi = (base + (intptr_t)(yhi + 1) * n2 * 4 + 15) & ~(intptr_t)15;
    const unsigned bytes = (unsigned)(hi - lo);
    mbar_expect_tx(bar, bytes + extra);
    bulk_load(slot + (lo - vo), reinterpret_cast<const void *>(lo), bytes, bar);
}

// Fine columns 2t - 2 .. 2t + 2 of a slot row into v[0 .. 4], by 8-byte
// loads of consecutive pairs (conflict-free across a warp): the row's first
// node sits at float fo of the slot, PAR = fo mod 2.  Columns -2 and -1
// (thread 0) are 0.  MASK (a row whose even columns are coarse nodes): the
// even columns 2t - 2 and 2t + 2 are not needed.  Every load stays inside
// the block's shared memory (the slots follow kSlabBarBytes of barriers).
template <int PAR, bool MASK>
__device__ __forceinline__ void slab_window(const float *slot, int fo, int t, float (&v)[5])
{
    const float2 *w = reinterpret_cast<const float2 *>(slot + fo - PAR) + t;
    if constexpr (PAR == 0) {  // pairs (2t-2, 2t-1), (2t, 2t+1), (2t+2, 2t+3)
        const float2 a = w[-1], b = w[0];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
        v[4] = MASK ? 0.f : w[1].x;
    } else {  // pairs (2t-3, 2t-2), (2t-1, 2t), (2t+1, 2t+2)
        const float2 b = w[0], c = w[1];
        v[0] = MASK ? 0.f : w[-1].y;
        v[1] = b.x;
        v[2] = b.y;
        v[3] = c.x;
        v[4] = c.y;
    }
    if (t == 0) v[0] = v[1] = 0.f;
}

// The dim-2 and dim-1 restriction of one fine plane from its slot into g[j]
// for the thread's coarse column t: EVEN = an even plane (its even rows hold
// coarse nodes, where C = 0; they are gathered into V when `gather`), P0 =
// the slot's element offset mod 2, KU = an interior band: every coarse row
// has the dim-1 stencil ku and every fine row it reads is inside the grid.
template <typename TW, int TY, bool EVEN, int P0, bool KU>
__device__ __forceinline__ void slab_plane(const float *slot, int s0, int n1, int n2, int Y0, int yown, int t,
                                           const float (&kx)[5], const float (&ku)[5],
                                           const float *__restrict__ k1, float (&g)[TY], bool gather,
                                           TW *__restrict__ vplane, int m2)
{
    constexpr int NR = SlabGeom<TY>::NR;
#pragma unroll
    for (int j = 0; j < TY; ++j) g[j] = 0.f;
    slab_for<0, NR>([&](auto RC) {
        constexpr int r = decltype(RC)::value;
        if (!KU) {
            const int y = 2 * Y0 - 2 + r;
            if (y < 0 || y >= n1) return;
        }
        // row parity = r parity (2 Y0 - 2 is even); the row's offset parity
        // is (s0 + r) mod 2 since n2 is odd
        constexpr bool MASK = EVEN && (r % 2 == 0);
        float v[5];
        slab_window<(P0 + r) & 1, MASK>(slot, s0 + r * n2, t, v);
        if (MASK && gather) {
            const int Yr = Y0 - 1 + r / 2;
            if (Yr >= yown && Yr < Y0 + TY) vplane[(int64_t)Yr * m2 + t] = static_cast<TW>(v[2]);
        }
        float h;
        if (MASK) {  // even columns of a coarse row are coarse nodes: C = 0
            h = fma_rn(kx[1], v[1], mul_rn(kx[3], v[3]));
        } else {
            h = fma_rn(kx[0], v[0], mul_rn(kx[1], v[1]));
            h = fma_rn(kx[2], v[2], h);
            h = fma_rn(kx[3], v[3], h);
            h = fma_rn(kx[4], v[4], h);
        }
        // fine row 2 Y0 - 2 + r feeds coarse row Y0 + j with tap r - 2 j
        slab_for<0, TY>([&](auto JC) {
            constexpr int j = decltype(JC)::value;
            constexpr int tap = r - 2 * j;
            if constexpr (tap >= 0 && tap <= 4) {
                const float ky = KU ? ku[tap] : __ldg(k1 + 5 * (Y0 + j) + tap);
                g[j] = fma_rn(ky, h, g[j]);
            }
        });
    });
}

template <typename TW, int TY, bool EVEN, bool KU>
__device__ __forceinline__ void slab_plane_p(int s0, const float *slot, int n1, int n2, int Y0, int yown, int t,
                                             const float (&kx)[5], const float (&ku)[5],
                                             const float *__restrict__ k1, float (&g)[TY], bool gather,
                                             TW *__restrict__ vplane, int m2)
{
    if (s0 & 1)
        slab_plane<TW, TY, EVEN, 1, KU>(slot, s0, n1, n2, Y0, yown, t, kx, ku, k1, g, gather, vplane, m2);
    else
        slab_plane<TW, TY, EVEN, 0, KU>(slot, s0, n1, n2, Y0, yown, t, kx, ku, k1, g, gather, vplane, m2);
}

// The final coarse column X = m2 - 1 of one fine plane, by the block's last
// warp after its main rows: lane r takes slot row r (its fine columns n2 - 3
// .. n2 - 1, the dim-2 stencil kxe), then lane j < TY sums the dim-1 stencil
// of coarse row Y0 + j over lanes 2j .. 2j + 4 by shuffles into *ge (lanes
// >= TY: unused).  Gathers the final coarse value of owned even rows into V.
template <typename TW, int TY, bool EVEN>
__device__ __forceinline__ float slab_last_col(const float *slot, int s0, int n1, int n2, int Y0, int yown, int lane,
                                               const float (&kxe)[5], bool ku_ok, const float (&ku)[5],
                                               const float *__restrict__ k1, bool gather, TW *__restrict__ vplane,
                                               int m2)
{
    constexpr int NR = SlabGeom<TY>::NR;
    float he = 0.f;
    const int y = 2 * Y0 - 2 + lane;
    if (lane < NR && y >= 0 && y < n1) {
        const float *row = slot + s0 + lane * n2 + (n2 - 3);
        const float a = row[0], b = row[1], c = row[2];
        const bool mask = EVEN && !(lane & 1);
        he = mask ? mul_rn(kxe[1], b) : fma_rn(kxe[2], c, fma_rn(kxe[0], a, mul_rn(kxe[1], b)));
        if (mask && gather) {
            const int Yr = Y0 - 1 + lane / 2;
            if (Yr >= yown && Yr < Y0 + TY) vplane[(int64_t)Yr * m2 + (m2 - 1)] = static_cast<TW>(c);
        }
    }
    float ge = 0.f;
#pragma unroll
    for (int tap = 0; tap < 5; ++tap) {
        const int src = 2 * lane + tap;
        const float hv = __shfl_sync(0xffffffffu, he, src & 31);
        if (lane < TY) {
            const float ky = ku_ok ? ku[tap] : __ldg(k1 + 5 * (Y0 + lane) + tap);
            ge = fma_rn(ky, hv, ge);
        }
    }
    return ge;
}

// The solve of M_{l-1} along dim 2 of row w of a finished coarse plane
// (srow, m2 = 32 C2 + 1 values; lane L holds nodes C2 L .. C2 L + C2 - 1,
// lane 31 also the final one), written back to srow and then to the F row
// by the warp in order (coalesced).
template <typename TW, int C2>
__device__ __forceinline__ void slab_xsolve_row(TW *srow, const TW *sfac, TW xa, TW xi, int lane, TW *frow)
{
    constexpr int M2 = 32 * C2 + 1;
    TW f[C2 + 1];
#pragma unroll
    for (int k = 0; k < C2; ++k) f[k] = srow[C2 * lane + k];
    f[C2] = (lane == 31) ? srow[32 * C2] : TW(0);
    rc_xsolve<TW, C2>(f, sfac, xa, xi, lane);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < C2; ++k) srow[C2 * lane + k] = f[k];
    if (lane == 31) srow[32 * C2] = f[C2];
    __syncwarp();
    for (int c = lane; c < M2; c += 32) frow[c] = srow[c];
}

// C2 = (m2 - 1) / 32 is the block's warp count: 1 .. 8 for blocks of up to
// 256 threads, 16 for 512
template <typename TW, int MAXT>
__device__ __forceinline__ void slab_xsolve_any(int c2, TW *srow, const TW *sfac, TW xa, TW xi, int lane, TW *frow)
{
    if constexpr (MAXT > 256) {
        slab_xsolve_row<TW, 16>(srow, sfac, xa, xi, lane, frow);
    } else {
        switch (c2) {
        case 1: slab_xsolve_row<TW, 1>(srow, sfac, xa, xi, lane, frow); break;
        case 2: slab_xsolve_row<TW, 2>(srow, sfac, xa, xi, lane, frow); break;
        case 4: slab_xsolve_row<TW, 4>(srow, sfac, xa, xi, lane, frow); break;
        default: slab_xsolve_row<TW, 8>(srow, sfac, xa, xi, lane, frow); break;
        }
    }
}

// One block per band x chunk item, (n2 - 1) / 2 = m2 - 1 <= MAXT threads:
// thread t owns coarse column t; the last warp also computes the final
// column m2 - 1 (lane j its coarse row Y0 + j).  MINB: blocks per SM the
// register allocation is sized for.  XS: each finished coarse plane's rows
// are solved along dim 2 (M_{l-1}, row j by warp j mod the warp count)
// before they are stored, so the host skips that dimension's solve.
template <typename TW, int TY, int MAXT, int MINB, bool XS>
__global__ void __launch_bounds__(MAXT, MINB) k_slab(SlabParams p)
{
    static_assert(2 * TY + 3 <= 32, "a band's fine rows fit one warp");
    extern __shared__ __align__(128) unsigned char slab_smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(slab_smem);
    unsigned char *ring = slab_smem + kSlabBarBytes;
    const float *__restrict__ A = static_cast<const float *>(p.A);
    TW *__restrict__ F = static_cast<TW *>(p.F);
    TW *__restrict__ V = static_cast<TW *>(p.V);
    const float *__restrict__ k0 = static_cast<const float *>(p.k0);
    const float *__restrict__ k1 = static_cast<const float *>(p.k1);
    const float *__restrict__ k2 = static_cast<const float *>(p.k2);
    const int t = threadIdx.x, lane = t & 31;
    const bool lastwarp = (t >> 5) == (int)(blockDim.x >> 5) - 1;
    const int n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2, NS = p.ns, SB = p.slot_bytes;
    const int64_t plane = (int64_t)n1 * n2, cplane = (int64_t)m1 * m2;
    const int w = t >> 5, C2 = (m2 - 1) / 32;
    // XS: two row buffers [TY][m2 + 1] and the dim-2 factor table [3][C2][32]
    TW *xrow = reinterpret_cast<TW *>(ring + (size_t)NS * SB);
    TW *xfac = xrow + 2 * TY * (m2 + 1);
    TW xa = TW(0), xi = TW(0);
    if constexpr (XS) {
        const TW *fx = static_cast<const TW *>(p.fx);
        for (int e = t; e < 3 * (m2 - 1); e += blockDim.x) {
            const int tt = e / (C2 * 32), k = (e / 32) % C2, l = e % 32;
            xfac[e] = fx[3 * (C2 * l + k) + tt];
        }
        xa = fx[3 * (m2 - 1)];
        xi = fx[3 * (m2 - 1) + 1];
    }

    // full[s] = bars[s] (the producer's arrival + the copy's bytes); empty[s]
    // = bars[NS + s] (one arrival per warp once it is done with the slot)
    __shared__ volatile int s_dead;  // a wait ran out: every warp leaves its loop
    const int nwarps = (int)(blockDim.x >> 5);
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&bars[s], 1);
            mbar_init(&bars[NS + s], (unsigned)nwarps);
        }
        mbar_init_fence();
        s_dead = 0;
    }
    __syncthreads();

    // dim-2 stencils of the thread's coarse column and of the final column
    // (fixed for the block)
    float kx[5], kxe[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        kx[s] = __ldg(k2 + 5 * t + s);
        kxe[s] = lastwarp ? __ldg(k2 + 5 * (m2 - 1) + s) : 0.f;
    }

    // producer (thread 0): the next position of the block's item sequence
    int p_item = blockIdx.x, p_z = 0, p_pos = 0;
    SlabItem p_it = {0, 0, 0, 0, 0, -1};
    if (p_item < p.nitems) {
        p_it = slab_item<TY>(p, p_item);
        p_z = p_it.zlo;
    }
    auto issue_next = [&]() {
        if (p_item >= p.nitems) return;
        const int s = p_pos % NS;
        if constexpr (!XS) {
            // the slot's previous use must be released by every warp
            if (p_pos >= NS && !mbar_wait(&bars[NS + s], (unsigned)((p_pos / NS - 1) & 1), p.wait_ns)) {
                s_dead = 1;
                return;
            }
        }
        slab_issue<TY>(A, plane, n1, n2, p_z, p_it.Y0, ring + (size_t)s * SB, &bars[s],
                       (p.hook && p_pos == 0) ? 16u : 0u);
        ++p_pos;
        if (++p_z > p_it.zhi) {
            p_item += gridDim.x;
            if (p_item < p.nitems) {
                p_it = slab_item<TY>(p, p_item);
                p_z = p_it.zlo;
            }
        }
    };
    // the predecessor on the stream (programmatic dependent launch) has
    // finished with the level array, F and V
    pdl_wait();
    if (t == 0)
        for (int s = 0; s < NS; ++s) issue_next();

    int pos = 0;
    bool dead = false;
    for (int item = blockIdx.x; item < p.nitems && !dead; item += gridDim.x) {
        const SlabItem it = slab_item<TY>(p, item);
        const int Y0 = it.Y0, yown = it.yown;
        // an interior band: one dim-1 stencil and every fine row inside the grid
        const bool ku_ok = p.kuni1 && Y0 >= 1 && Y0 + TY <= m1 - 1;
        float ku[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) ku[s] = ku_ok ? __ldg(k1 + 5 * Y0 + s) : 0.f;

        // rolling plane accumulators (coarse planes Z - 1, Z, Z + 1) of
        // column t, and of the final column in lane j < TY of the last warp
        float accP[TY], accC[TY], accN[TY], eP = 0.f, eC = 0.f, eN = 0.f;
#pragma unroll
        for (int j = 0; j < TY; ++j) accP[j] = accC[j] = accN[j] = 0.f;
        // F rows of coarse plane Zo: stored (or, XS, put in the row buffer of
        // Zo's parity, solved and stored by warp j after the next barrier)
        int pend = -1;  // XS: the plane whose rows wait for their solve
        auto store = [&](int Zo) {
            if constexpr (XS) {
                TW *xr = xrow + (Zo & 1) * TY * (m2 + 1);
#pragma unroll
                for (int j = 0; j < TY; ++j) xr[j * (m2 + 1) + t] = static_cast<TW>(accP[j]);
                if (lastwarp && lane < TY) xr[lane * (m2 + 1) + (m2 - 1)] = static_cast<TW>(eP);
                pend = Zo;
            } else {
                TW *f = F + (int64_t)Zo * cplane + (int64_t)Y0 * m2;
#pragma unroll
                for (int j = 0; j < TY; ++j)
                    if (Y0 + j >= yown) f[(int64_t)j * m2 + t] = static_cast<TW>(accP[j]);
                if (lastwarp && lane < TY && Y0 + lane >= yown)
                    f[(int64_t)lane * m2 + (m2 - 1)] = static_cast<TW>(eP);
            }
        };
        auto solve_pending = [&]() {
            if constexpr (XS) {
                if (pend >= 0) {
                    // row j by warp j mod (warps of the block)
                    for (int j = w; j < TY; j += (int)(blockDim.x >> 5))
                        if (Y0 + j >= yown)
                            slab_xsolve_any<TW, MAXT>(C2, xrow + (pend & 1) * TY * (m2 + 1) + j * (m2 + 1), xfac, xa,
                                                      xi, lane, F + (int64_t)pend * cplane + (int64_t)(Y0 + j) * m2);
                }
                pend = -1;
            }
        };

        for (int z = it.zlo; z <= it.zhi; ++z, ++pos) {
            const int s = pos % NS;
            const bool ok = mbar_wait(&bars[s], (unsigned)((pos / NS) & 1), p.wait_ns);
            const float *slot = reinterpret_cast<const float *>(ring + (size_t)s * SB);
            const int s0 = slab_s0(A, plane, n2, z, Y0);
            float g[TY], ge = 0.f;
            const int Z = z >> 1;
            if (z & 1) {
                // odd plane 2Z + 1: tap 3 of coarse plane Z, tap 1 of Z + 1
                // (accP holds plane Z, accC plane Z + 1)
                if (ku_ok)
                    slab_plane_p<TW, TY, false, true>(s0, slot, n1, n2, Y0, yown, t, kx, ku, k1, g, false, V, m2);
                else
                    slab_plane_p<TW, TY, false, false>(s0, slot, n1, n2, Y0, yown, t, kx, ku, k1, g, false, V, m2);
                if (lastwarp)
                    ge = slab_last_col<TW, TY, false>(slot, s0, n1, n2, Y0, yown, lane, kxe, ku_ok, ku, k1, false, V,
                                                      m2);
                const float kP = __ldg(k0 + 5 * Z + 3), kC = __ldg(k0 + 5 * (Z + 1) + 1);
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accP[j] = fma_rn(kP, g[j], accP[j]);
                    accC[j] = fma_rn(kC, g[j], accC[j]);
                }
                eP = fma_rn(kP, ge, eP);
                eC = fma_rn(kC, ge, eC);
            } else {
                // even plane 2Z: tap 4 of Z - 1, tap 2 of Z, tap 0 of Z + 1 (accP
                // holds coarse plane Z - 1, accC plane Z)
                const bool own = Z >= it.Zs && Z < it.Ze;
                TW *vplane = V + (int64_t)Z * cplane;
                if (ku_ok)
                    slab_plane_p<TW, TY, true, true>(s0, slot, n1, n2, Y0, yown, t, kx, ku, k1, g, own, vplane, m2);
                else
                    slab_plane_p<TW, TY, true, false>(s0, slot, n1, n2, Y0, yown, t, kx, ku, k1, g, own, vplane, m2);
                if (lastwarp)
                    ge = slab_last_col<TW, TY, true>(slot, s0, n1, n2, Y0, yown, lane, kxe, ku_ok, ku, k1, own,
                                                     vplane, m2);
                const float kP = (Z >= 1) ? __ldg(k0 + 5 * (Z - 1) + 4) : 0.f;
                const float kC = __ldg(k0 + 5 * Z + 2);
                const float kN = (Z + 1 < m0) ? __ldg(k0 + 5 * (Z + 1)) : 0.f;
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accP[j] = fma_rn(kP, g[j], accP[j]);
                    accC[j] = fma_rn(kC, g[j], accC[j]);
                    accN[j] = mul_rn(kN, g[j]);
                }
                eP = fma_rn(kP, ge, eP);
                eC = fma_rn(kC, ge, eC);
                eN = mul_rn(kN, ge);
                // F(Z - 1) is complete once the planes up to 2Z are in
                if (Z - 1 >= it.Zs && Z - 1 < it.Ze) store(Z - 1);
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accP[j] = accC[j];
                    accC[j] = accN[j];
                }
                eP = eC;
                eC = eN;
            }
            if constexpr (XS) {
                // every thread is done with slot s (and agrees on whether a
                // wait ran out) before it is refilled
                if (__syncthreads_or(!ok)) {
                    dead = true;
                    break;
                }
                if (t == 0) issue_next();
                solve_pending();  // the rows stored before this barrier
            } else {
                // the warp releases slot s; thread 0 refills the slot of the
                // position NS ahead once every warp has released it, while
                // the other warps go on with the next staged plane
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[NS + s]);
                if (!ok) s_dead = 1;
                if (t == 0 && !s_dead) issue_next();
                if (s_dead) {
                    dead = true;
                    break;
                }
            }
        }
        // the last coarse plane of the grid has no contributions beyond it
        // (after the final shift it is in accP)
        if (!dead && it.zhi == 2 * (m0 - 1) && m0 - 1 >= it.Zs && m0 - 1 < it.Ze) {
            store(m0 - 1);
            if constexpr (XS) {
                __syncthreads();
                solve_pending();
            }
        }
    }
    if constexpr (XS) {
        if (dead) {
            // record it, then let the copies this block issued (from the one
            // whose wait ran out on) land, bounded, before its shared memory
            // goes away
            if (t == 0) {
                atomicOr(p.status, 1u);
                for (int e = pos; e < p_pos; ++e) (void)mbar_wait(&bars[e % NS], (unsigned)((e / NS) & 1), p.wait_ns);
            }
            __syncthreads();
        }
    } else {
        // the warps leave their loops independently; a block where a wait ran
        // out records it and lets the copies it issued last (one per slot;
        // earlier ones were consumed) land, bounded, before its shared memory
        // goes away
        if (t == 0 && s_dead) {
            atomicOr(p.status, 1u);
            for (int e = max(0, p_pos - NS); e < p_pos; ++e)
                (void)mbar_wait(&bars[e % NS], (unsigned)((e / NS) & 1), p.wait_ns);
        }
        __syncthreads();
    }
}

}  // namespace mg
