// persist.cuh -- many independent fields refactored by one persistent launch.
//
// The level steps are those of Section II-A (Eq. 1-2) as organised for the
// GPU in Section III-A: coefficients by interpolation, the load vector by the
// stencils K = P^T M_l along each dimension, the correction by the
// tridiagonal solves M_{l-1} z = F along each dimension, V += z; the
// recomposition mirrors them.  The solves along different dimensions act on
// different tensor factors and commute, as do the stencils, so each level is
// cut into tasks whose items are independent:
//   A  fine plane(s) i0: coefficients written in place (decomposition), the
//      plane's coarse nodes gathered into V, and G = (K_1 (x) K_2) C, one row
//      of K_2 C per fine row kept in a ring of the block
//   C  a panel of 32 lines along dim 0: F = K_0 G (the G rows of the panel
//      streamed through a ring), then the solve along dim 0
//   B  coarse plane(s) Z: the solves along dims 2 and 1, then V += z
//      (decomposition) or z into F (recomposition)
//   D  fine plane(s) i0 (recomposition): U = C + Pi (V - z)
// plus the levels of a small array in one block (small.cuh) and the final
// placement of every level's coarse values.  Fields with two active dims are
// relabelled (rows, 1, columns): their rows are the planes, several to an
// item, one per warp.  Each warp copies the rows it needs next into shared
// memory with cp.async while it computes on the current ones.
//
// The blocks of the grid take items from a queue (an atomic head over an
// item list the host ordered by a list-scheduling model).  A task's items
// wait, bounded, until every item of the tasks it depends on is done; the
// list puts those earlier, so an item only ever waits for items that blocks
// already hold, and the launch needs no co-residency.  A wait that runs out
// sets a status bit and the block goes on.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "params.h"
#include "persist_params.h"
#include "small.cuh"

namespace mg {

__device__ __forceinline__ unsigned persist_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename TW>
struct PGeo {
    int n0, n1, n2, m0, m1, m2;
    int c0, c1, c2;  // the dim coarsens at this level
    const TW *w0, *w1, *w2, *k0, *k1, *k2, *f0, *f1, *f2;
};

template <typename TW>
__device__ __forceinline__ PGeo<TW> pgeo(const PersistLevel &L)
{
    PGeo<TW> g;
    g.n0 = L.n[0]; g.n1 = L.n[1]; g.n2 = L.n[2];
    g.m0 = L.m[0]; g.m1 = L.m[1]; g.m2 = L.m[2];
    g.c0 = L.co[0]; g.c1 = L.co[1]; g.c2 = L.co[2];
    g.w0 = static_cast<const TW *>(L.w[0]); g.w1 = static_cast<const TW *>(L.w[1]);
    g.w2 = static_cast<const TW *>(L.w[2]);
    g.k0 = static_cast<const TW *>(L.k[0]); g.k1 = static_cast<const TW *>(L.k[1]);
    g.k2 = static_cast<const TW *>(L.k[2]);
    g.f0 = static_cast<const TW *>(L.fac[0]); g.f1 = static_cast<const TW *>(L.fac[1]);
    g.f2 = static_cast<const TW *>(L.fac[2]);
    return g;
}

__host__ __device__ __forceinline__ int persist_round4(int x) { return (x + 3) & ~3; }

// Block-wide copy of a table into shared memory (read-only data).
template <typename TW>
__device__ __forceinline__ void persist_table(TW *dst, const TW *src, int n)
{
    for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = __ldg(src + e);
}

// n elements at stride s from global into shared memory (cp.async, one
// element per copy, coalesced across the warp for s = 1); the caller commits
// and waits.
template <typename T>
__device__ __forceinline__ void persist_stage(T *dst, const T *src, int n, int s, int lane)
{
    for (int i = lane; i < n; i += 32) cp_async_elem<T>(dst + i, src + (int64_t)i * s, true);
}

// Elements 2j and 2j+1 of a shared-memory row (8- or 16-byte aligned pair).
template <typename T>
struct Pair2 {
    using V = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    static __device__ __forceinline__ void load(const T *row, int j, T &a, T &b)
    {
        const V v = reinterpret_cast<const V *>(row)[j];
        a = static_cast<T>(v.x);
        b = static_cast<T>(v.y);
    }
    static __device__ __forceinline__ void store(T *row, int j, T a, T b)
    {
        V v;
        v.x = a;
        v.y = b;
        reinterpret_cast<V *>(row)[j] = v;
    }
};

// ---------------------------------------------------------------------------
// Shared-memory layouts (elements of TW), shared with the host, which sizes
// the launch by the largest item of the batch.  rn / rm: a fine / coarse row
// rounded up to four elements; pm: the level runs by planes (dim 1 coarsens).
// ---------------------------------------------------------------------------
struct PersistSmem {
    // phase A: tables w1, w2, k1, k2; the ring of K_2 C rows (active dim 1);
    // per warp (active dim 1) two coarse rows of the plane's coarse grid W
    // and two sets of {two fine rows, four coarse source rows}, or one row
    // of W, one fine row and two coarse source rows
    static __host__ __device__ int a_tab(int n1, int n2, int m1, int m2)
    {
        return persist_round4(2 * n1 + 2 * n2 + 5 * m1 + 5 * m2);
    }
    static __host__ __device__ int a_ring(int pm, int m2) { return pm ? kPersistRing * persist_round4(m2) : 0; }
    static __host__ __device__ int a_warp(int pm, int n2, int m2)
    {
        const int rn = persist_round4(n2), rm = persist_round4(m2);
        return pm ? 2 * rm + 4 * rn + 8 * rm : rm + rn + 2 * rm;
    }
    static __host__ __device__ int64_t a(int pm, int n1, int n2, int m1, int m2)
    {
        return a_tab(n1, n2, m1, m2) + a_ring(pm, m2) + (int64_t)kPersistWarps * a_warp(pm, n2, m2);
    }
    // phase B: factors of dims 2 and 1, then the coarse plane (active dim 1)
    // or one coarse row per warp
    static __host__ __device__ int b_tab(int m1, int m2) { return persist_round4(3 * m1 + 3 * m2); }
    static __host__ __device__ int64_t b(int pm, int m1, int m2)
    {
        return b_tab(m1, m2) + (pm ? (int64_t)m1 * m2 : (int64_t)kPersistWarps * persist_round4(m2));
    }
    // phase C: factors of dim 0, the panel of F, the ring of G rows, four
    // carry arrays
    static __host__ __device__ int c_tab(int m0) { return persist_round4(3 * m0); }
    static __host__ __device__ int64_t c(int m0)
    {
        return c_tab(m0) + ((int64_t)m0 + kPersistGRing + 4 * kPersistWarps) * kPersistPanel;
    }
    // phase D: tables w1, w2; per warp (active dim 1) two rows of W and two
    // sets of {two fine rows, four coarse source rows of V and z}, or one
    // fine row and four source rows
    static __host__ __device__ int d_tab(int n1, int n2) { return persist_round4(2 * n1 + 2 * n2); }
    static __host__ __device__ int d_warp(int pm, int n2, int m2)
    {
        const int rn = persist_round4(n2), rm = persist_round4(m2);
        return pm ? 2 * rm + 4 * rn + 8 * rm : rn + 4 * rm;
    }
    static __host__ __device__ int64_t d(int pm, int n1, int n2, int m2)
    {
        return d_tab(n1, n2) + (int64_t)kPersistWarps * d_warp(pm, n2, m2);
    }
};

// ---------------------------------------------------------------------------
// Phase A
// ---------------------------------------------------------------------------

// Fine row i1 of plane i0 by one warp, staged in rb: (decomposition) its
// coefficients C = U - Pi U on the nodes outside the coarse grid, written in
// place to xrow and rb; the coarse nodes counted as 0 in rb; then
// H(X) = sum_c K_2[X][c] C(2X - 2 + c) into hrow (m2 values).
// c0 / c1: coarse rows i1/2 and i1/2 + (i1 odd) of the plane.
template <typename XT, typename TW, int MODE>
__device__ __forceinline__ void persist_a_row(const PGeo<TW> &g, XT *xrow, int i1, bool podd, const TW *tw1,
                                              const TW *tw2, const TW *tk2, const TW *c0, const TW *c1, XT *rb,
                                              TW *hrow, int lane)
{
    const int q1 = g.c1 & i1 & 1;
    const bool rodd = podd || q1;  // every node of the row is outside the coarse grid
    if (g.c2) {
        // lane takes the column pairs (2j, 2j+1): both read coarse nodes j
        // (and j+1), the even column only when the row is odd
        const int np2 = (g.n2 + 1) >> 1;
        for (int j = lane; j < np2; j += 32) {
            const bool ho = 2 * j + 1 < g.n2;
            XT ue, uo;
            if (ho) {
                Pair2<XT>::load(rb, j, ue, uo);
            } else {
                ue = rb[2 * j];
                uo = XT(0);
            }
            XT ce = XT(0), co = uo;
            if constexpr (MODE == MODE_DEC) {
                const TW a0 = c0[j];
                const TW wl1 = q1 ? tw1[2 * i1] : TW(1), wr1 = q1 ? tw1[2 * i1 + 1] : TW(0);
                const TW a1 = q1 ? c1[j] : a0;
                if (rodd) {
                    ce = static_cast<XT>(static_cast<TW>(ue) - (wl1 * a0 + wr1 * a1));
                    xrow[2 * j] = ce;
                }
                if (ho) {
                    TW wl2, wr2;
                    Pair2<TW>::load(tw2, 2 * j + 1, wl2, wr2);
                    const TW b0 = c0[j + 1], b1 = q1 ? c1[j + 1] : b0;
                    const TW x0 = wl2 * a0 + wr2 * b0, x1 = wl2 * a1 + wr2 * b1;
                    co = static_cast<XT>(static_cast<TW>(uo) - (wl1 * x0 + wr1 * x1));
                    xrow[2 * j + 1] = co;
                }
            } else {
                if (rodd) ce = ue;
            }
            if (ho) Pair2<XT>::store(rb, j, ce, co);
            else rb[2 * j] = ce;
        }
        __syncwarp();
        for (int X = lane; X < g.m2; X += 32) {
            TW h = tk2[5 * X + 2] * static_cast<TW>(rb[2 * X]);
            if (X > 0) {
                XT r0, r1;
                Pair2<XT>::load(rb, X - 1, r0, r1);
                h += tk2[5 * X] * static_cast<TW>(r0) + tk2[5 * X + 1] * static_cast<TW>(r1);
            }
            if (2 * X + 1 < g.n2) {
                h += tk2[5 * X + 3] * static_cast<TW>(rb[2 * X + 1]) + tk2[5 * X + 4] * static_cast<TW>(rb[2 * X + 2]);
            }
            hrow[X] = h;
        }
        __syncwarp();
        return;
    }
    // P = I along dim 2: the row's own nodes, its stencil and solve cancel
    if constexpr (MODE == MODE_DEC) {
        const TW wl1 = q1 ? tw1[2 * i1] : TW(1), wr1 = q1 ? tw1[2 * i1 + 1] : TW(0);
        for (int i2 = lane; i2 < g.n2; i2 += 32) {
            if (rodd) {
                const XT c = static_cast<XT>(static_cast<TW>(rb[i2]) - (wl1 * c0[i2] + wr1 * c1[i2]));
                xrow[i2] = c;
                rb[i2] = c;
            } else {
                rb[i2] = XT(0);
            }
        }
    } else {
        for (int i2 = lane; i2 < g.n2; i2 += 32)
            if (!rodd) rb[i2] = XT(0);
    }
    __syncwarp();
    for (int X = lane; X < g.m2; X += 32) hrow[X] = static_cast<TW>(rb[X]);
    __syncwarp();
}

template <typename XT, typename TW, int MODE>
__device__ void persist_a(const PersistLevel &L, int item, int per, TW *sm)
{
    const PGeo<TW> g = pgeo<TW>(L);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t np = (int64_t)g.n1 * g.n2, mc = (int64_t)g.m1 * g.m2;
    const int rn = persist_round4(g.n2), rm = persist_round4(g.m2);
    const int sx = g.c2 ? 2 : 1;  // stride of the coarse nodes along a fine row
    XT *X = static_cast<XT *>(L.X);
    TW *V = static_cast<TW *>(L.V), *G = static_cast<TW *>(L.G);
    TW *tw1 = sm, *tw2 = tw1 + 2 * g.n1, *tk1 = tw2 + 2 * g.n2, *tk2 = tk1 + 5 * g.m1;
    TW *ring = sm + PersistSmem::a_tab(g.n1, g.n2, g.m1, g.m2);
    TW *wb = ring + PersistSmem::a_ring(g.c1, g.m2) + warp * PersistSmem::a_warp(g.c1, g.n2, g.m2);
    TW *wrow0 = wb, *wrow1 = wb + rm;

    if (!g.c1) {
        // by rows: row r = item * per + warp of the n0 x n1 rows (its own
        // coarse row: dim 1 does not coarsen); the row and (odd plane of a
        // decomposition) its neighbours' coarse nodes staged
        const int r = item * per + warp;
        const bool mine = warp < per && r < g.n0 * g.n1;
        const int i0 = mine ? r / g.n1 : 0, i1 = mine ? r % g.n1 : 0;
        const bool podd = g.c0 && (i0 & 1);
        const int64_t ro = (int64_t)i0 * np + (int64_t)i1 * g.n2;
        XT *rb = reinterpret_cast<XT *>(wb + rm);
        XT *sa = reinterpret_cast<XT *>(wb + rm + rn), *sb = reinterpret_cast<XT *>(wb + 2 * rm + rn);
        if (mine) {
            persist_stage<XT>(rb, X + ro, g.n2, 1, lane);
            if (MODE == MODE_DEC && podd) {
                persist_stage<XT>(sa, X + ro - np, g.m2, sx, lane);
                persist_stage<XT>(sb, X + ro + np, g.m2, sx, lane);
            }
        }
        cp_async_commit();
        if (g.c2) {
            persist_table<TW>(tw2, g.w2, 2 * g.n2);
            persist_table<TW>(tk2, g.k2, 5 * g.m2);
        }
        cp_async_wait<0>();
        __syncthreads();  // the tables
        if (mine) {
            const TW wl = podd ? __ldg(g.w0 + 2 * i0) : TW(0), wr = podd ? __ldg(g.w0 + 2 * i0 + 1) : TW(0);
            TW *Vr = V + (int64_t)(i0 >> g.c0) * mc + (int64_t)i1 * g.m2;
            for (int x = lane; x < g.m2; x += 32) {
                if (podd) {
                    if (MODE == MODE_DEC) wrow0[x] = wl * static_cast<TW>(sa[x]) + wr * static_cast<TW>(sb[x]);
                } else {
                    const TW v = static_cast<TW>(rb[sx * x]);
                    wrow0[x] = v;
                    Vr[x] = v;
                }
            }
            __syncwarp();
            persist_a_row<XT, TW, MODE>(g, X + ro, i1, podd, tw1, tw2, tk2, wrow0, wrow0, rb,
                                        G + (int64_t)i0 * mc + (int64_t)i1 * g.m2, lane);
        }
        return;
    }

    // a plane with an active dim 1: warps take pairs of fine rows (2Y, 2Y+1)
    // eight at a time, the next pair's rows (and the coarse rows its
    // interpolation needs) staged while the current pair is computed; the
    // K_2 C rows go to the ring (row r at slot r % 32), and G row
    // Y' = (pair batch start) - 1 + warp is reduced along dim 1 once the
    // rows 2Y' - 2 .. 2Y' + 2 are in the ring
    const int i0 = item;
    const bool podd = g.c0 && (i0 & 1);
    const TW wl = podd ? __ldg(g.w0 + 2 * i0) : TW(0), wr = podd ? __ldg(g.w0 + 2 * i0 + 1) : TW(0);
    TW *sets = wb + 2 * rm;
    XT *Xp = X + (int64_t)i0 * np;
    TW *Gp = G + (int64_t)i0 * mc;
    TW *Vp = V + (int64_t)(i0 >> g.c0) * mc;
    auto row = [&](int set, int k) { return reinterpret_cast<XT *>(sets + set * (2 * rn + 4 * rm) + k * rn); };
    auto src = [&](int set, int k) {
        return reinterpret_cast<XT *>(sets + set * (2 * rn + 4 * rm) + 2 * rn + k * rm);
    };
    // sources of W: even plane: row 2Y+2's coarse nodes (row 2Y's are in the
    // staged row itself); odd plane: rows 2Y and 2Y+2 of planes i0 -+ 1
    auto stage_pair = [&](int Y, int set) {
        if (Y < g.m1) {
            const bool two = 2 * Y + 1 < g.n1;
            persist_stage<XT>(row(set, 0), Xp + (int64_t)(2 * Y) * g.n2, g.n2, 1, lane);
            if (two) persist_stage<XT>(row(set, 1), Xp + (int64_t)(2 * Y + 1) * g.n2, g.n2, 1, lane);
            if (MODE == MODE_DEC) {
                if (!podd) {
                    if (two) persist_stage<XT>(src(set, 0), Xp + (int64_t)(2 * Y + 2) * g.n2, g.m2, sx, lane);
                } else {
                    const XT *pa = Xp - np, *pb = Xp + np;
                    persist_stage<XT>(src(set, 0), pa + (int64_t)(2 * Y) * g.n2, g.m2, sx, lane);
                    persist_stage<XT>(src(set, 1), pb + (int64_t)(2 * Y) * g.n2, g.m2, sx, lane);
                    if (two) {
                        persist_stage<XT>(src(set, 2), pa + (int64_t)(2 * Y + 2) * g.n2, g.m2, sx, lane);
                        persist_stage<XT>(src(set, 3), pb + (int64_t)(2 * Y + 2) * g.n2, g.m2, sx, lane);
                    }
                }
            }
        }
        cp_async_commit();
    };
    stage_pair(warp, 0);
    persist_table<TW>(tw1, g.w1, 2 * g.n1);
    persist_table<TW>(tk1, g.k1, 5 * g.m1);
    if (g.c2) {
        persist_table<TW>(tw2, g.w2, 2 * g.n2);
        persist_table<TW>(tk2, g.k2, 5 * g.m2);
    }
    __syncthreads();  // the tables
    for (int b0 = 0, set = 0; b0 <= g.m1; b0 += kPersistWarps, set ^= 1) {
        const int Y = b0 + warp;
        stage_pair(Y + kPersistWarps, set ^ 1);
        if (Y < g.m1) {
            const bool two = 2 * Y + 1 < g.n1;
            cp_async_wait<1>();  // this pair's copies (the next pair's may still be in flight)
            __syncwarp();
            XT *r0 = row(set, 0);
            // coarse rows Y and Y+1 of the plane's coarse grid; the even
            // plane's row Y also into V
            for (int x = lane; x < g.m2; x += 32) {
                if (!podd) {
                    const TW v = static_cast<TW>(r0[sx * x]);
                    wrow0[x] = v;
                    Vp[(int64_t)Y * g.m2 + x] = v;
                    if (MODE == MODE_DEC && two) wrow1[x] = static_cast<TW>(src(set, 0)[x]);
                } else if (MODE == MODE_DEC) {
                    wrow0[x] = wl * static_cast<TW>(src(set, 0)[x]) + wr * static_cast<TW>(src(set, 1)[x]);
                    if (two) wrow1[x] = wl * static_cast<TW>(src(set, 2)[x]) + wr * static_cast<TW>(src(set, 3)[x]);
                }
            }
            __syncwarp();
            persist_a_row<XT, TW, MODE>(g, Xp + (int64_t)(2 * Y) * g.n2, 2 * Y, podd, tw1, tw2, tk2, wrow0, wrow0,
                                        r0, ring + ((2 * Y) & (kPersistRing - 1)) * rm, lane);
            if (two)
                persist_a_row<XT, TW, MODE>(g, Xp + (int64_t)(2 * Y + 1) * g.n2, 2 * Y + 1, podd, tw1, tw2, tk2,
                                            wrow0, wrow1, row(set, 1), ring + ((2 * Y + 1) & (kPersistRing - 1)) * rm,
                                            lane);
        }
        __syncthreads();
        const int Yg = b0 - 1 + warp;
        if (Yg >= 0 && Yg < g.m1) {
            TW k[5];
            const TW *r[5];
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const int i1 = 2 * Yg - 2 + b;
                const bool ok = i1 >= 0 && i1 < g.n1;
                k[b] = ok ? tk1[5 * Yg + b] : TW(0);
                r[b] = ring + ((ok ? i1 : 0) & (kPersistRing - 1)) * rm;
            }
            for (int x = lane; x < g.m2; x += 32) {
                TW v = TW(0);
#pragma unroll
                for (int b = 0; b < 5; ++b) v += k[b] * r[b][x];
                Gp[(int64_t)Yg * g.m2 + x] = v;
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Phase C: a panel of up to 32 lines along dim 0 (coarse row Y, columns
// x0 .. x0 + 31), lane = line.  F = K_0 G, coarse plane Z by warp Z % 8,
// the G rows streamed through a ring; then the solve, warp w taking nodes
// [w ch, w ch + ch) of every line, the chunk carries composed through
// shared memory; F back.
// ---------------------------------------------------------------------------
template <typename TW>
__device__ void persist_c(const PersistLevel &L, int item, TW *sm)
{
    const PGeo<TW> g = pgeo<TW>(L);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kPersistWarps, PW = kPersistPanel, RG = kPersistGRing;
    const int npan = (g.m2 + PW - 1) / PW;
    const int Y = item / npan, x0 = (item % npan) * PW;
    const int x = x0 + lane;
    const bool xok = x < g.m2;
    const int64_t rs = (int64_t)g.m1 * g.m2;
    TW *F = static_cast<TW *>(L.F);
    const TW *G = static_cast<const TW *>(L.G);
    const int64_t base = (int64_t)Y * g.m2 + x;
    TW *tf0 = sm;
    TW *S = sm + PersistSmem::c_tab(g.m0);
    TW *ring = S + (int64_t)g.m0 * PW;
    TW *cy = ring + RG * PW, *cp = cy + NW * PW, *cz = cp + NW * PW, *cq = cz + NW * PW;
    if (!g.c0) {  // P = I along dim 0 (m0 = n0): F is G
        if (xok)
            for (int Z = warp; Z < g.m0; Z += NW) F[Z * rs + base] = G[Z * rs + base];
        return;
    }
    // G row r of the panel into ring slot r % RG (zero-filled past the last
    // column); rows past the level are skipped
    auto stage_row = [&](int r) {
        if (r < g.n0) cp_async_elem<TW>(ring + (r & (RG - 1)) * PW + lane, xok ? G + r * rs + base : G, xok);
    };
    // rows 0 .. 2 NW: those of the first NW coarse planes (2 per warp, warp 0
    // also row 2 NW), then the next group's 2 NW rows; per group of NW
    // planes the rows two groups ahead (the ring spans the rows read by the
    // slowest warp and those copied by the fastest)
    stage_row(2 * warp);
    stage_row(2 * warp + 1);
    if (warp == 0) stage_row(2 * NW);
    cp_async_commit();
    stage_row(2 * NW + 1 + 2 * warp);
    stage_row(2 * NW + 2 + 2 * warp);
    cp_async_commit();
    persist_table<TW>(tf0, g.f0, 3 * g.m0);
    for (int z0 = 0; z0 < g.m0; z0 += NW) {
        // rows 2 z0 + 4 NW + 1 .. 2 z0 + 6 NW: the group after next
        const int nx = 2 * z0 + 4 * NW + 1;
        stage_row(nx + 2 * warp);
        stage_row(nx + 2 * warp + 1);
        cp_async_commit();
        cp_async_wait<2>();
        __syncthreads();
        const int Z = z0 + warp;
        if (Z < g.m0) {
            TW f = TW(0);
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const int i0 = 2 * Z - 2 + a;
                if (i0 >= 0 && i0 < g.n0) f += __ldg(g.k0 + 5 * Z + a) * ring[(i0 & (RG - 1)) * PW + lane];
            }
            S[Z * PW + lane] = f;
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    const int ch = (g.m0 + NW - 1) / NW;
    const int s = min(g.m0, warp * ch), e = min(g.m0, s + ch);
    // forward, local from a zero carry
    TW t = TW(0), P = TW(1);
    for (int i = s; i < e; ++i) {
        const TW a = tf0[3 * i];
        t = S[i * PW + lane] - a * t;
        S[i * PW + lane] = t;
        P *= -a;
    }
    cy[warp * PW + lane] = t;
    cp[warp * PW + lane] = P;
    __syncthreads();
    TW c = TW(0);
    for (int w = 0; w < warp; ++w) c = cy[w * PW + lane] + cp[w * PW + lane] * c;
    TW Pf = TW(1);
    for (int i = s; i < e; ++i) {
        Pf *= -tf0[3 * i];
        S[i * PW + lane] += Pf * c;
    }
    // backward, local from a zero carry
    t = TW(0);
    TW Q = TW(1);
    for (int i = e - 1; i >= s; --i) {
        const TW q = tf0[3 * i + 2];
        t = tf0[3 * i + 1] * S[i * PW + lane] - q * t;
        S[i * PW + lane] = t;
        Q *= -q;
    }
    cz[warp * PW + lane] = t;
    cq[warp * PW + lane] = Q;
    __syncthreads();
    TW d = TW(0);
    for (int w = NW - 1; w > warp; --w) d = cz[w * PW + lane] + cq[w * PW + lane] * d;
    TW Qb = TW(1);
    for (int i = e - 1; i >= s; --i) {
        Qb *= -tf0[3 * i + 2];
        S[i * PW + lane] += Qb * d;
    }
    __syncthreads();
    if (xok)
        for (int Z = warp; Z < g.m0; Z += NW) F[Z * rs + base] = S[Z * PW + lane];
}

// ---------------------------------------------------------------------------
// Phase B: the solves along dims 2 and 1 of coarse plane(s) Z, then
// V += z (decomposition) or z back into F (recomposition).
// ---------------------------------------------------------------------------

// M z = f along one line of m nodes at stride s in shared memory, by one
// thread (the Thomas recurrences of the tabulated factors).
template <typename TW>
__device__ __noinline__ void persist_line_solve(TW *f, int s, int m, const TW *fac)
{
    TW t = TW(0);
    for (int i = 0; i < m; ++i) {
        t = f[i * s] - fac[3 * i] * t;
        f[i * s] = t;
    }
    t = TW(0);
    for (int i = m - 1; i >= 0; --i) {
        t = fac[3 * i + 1] * f[i * s] - fac[3 * i + 2] * t;
        f[i * s] = t;
    }
}

// M z = f along one line of m nodes in shared memory by one warp: lane L
// owns nodes [L C, L C + C), C = ceil(m / 32).  Each lane runs the forward
// recurrence y_i = f_i - a_i y_{i-1} over its chunk from a zero carry, the
// chunks' affine maps (carry -> chunk-end value) are composed by a warp
// scan, and each lane adds the true carry times the running product of
// (-a_i); the backward recurrence z_i = inv_i y_i - q_i z_{i+1} likewise
// from the right.
template <typename TW>
__device__ __forceinline__ void persist_warp_solve(TW *f, int m, const TW *fac, int lane)
{
    const int C = (m + 31) >> 5;
    const int s = min(m, lane * C), e = min(m, s + C);
    TW t = TW(0), P = TW(1);
    for (int i = s; i < e; ++i) {
        const TW a = fac[3 * i];
        t = f[i] - a * t;
        f[i] = t;
        P *= -a;
    }
    TW Pi = P, yi = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const TW Pu = __shfl_up_sync(0xffffffffu, Pi, o), yu = __shfl_up_sync(0xffffffffu, yi, o);
        if (lane >= o) {
            yi = yi + Pi * yu;
            Pi = Pi * Pu;
        }
    }
    TW c = __shfl_up_sync(0xffffffffu, yi, 1);
    if (lane == 0) c = TW(0);
    TW Pf = TW(1);
    for (int i = s; i < e; ++i) {
        Pf *= -fac[3 * i];
        f[i] += Pf * c;
    }
    t = TW(0);
    TW Q = TW(1);
    for (int i = e - 1; i >= s; --i) {
        const TW q = fac[3 * i + 2];
        t = fac[3 * i + 1] * f[i] - q * t;
        f[i] = t;
        Q *= -q;
    }
    TW Qi = Q, zi = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const TW Qd = __shfl_down_sync(0xffffffffu, Qi, o), zd = __shfl_down_sync(0xffffffffu, zi, o);
        if (lane + o < 32) {
            zi = zi + Qi * zd;
            Qi = Qi * Qd;
        }
    }
    TW d = __shfl_down_sync(0xffffffffu, zi, 1);
    if (lane == 31) d = TW(0);
    TW Qb = TW(1);
    for (int i = e - 1; i >= s; --i) {
        Qb *= -fac[3 * i + 2];
        f[i] += Qb * d;
    }
    __syncwarp();
}

template <typename TW, int MODE>
__device__ void persist_b(const PersistLevel &L, int item, int per, TW *sm)
{
    const PGeo<TW> g = pgeo<TW>(L);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t mc = (int64_t)g.m1 * g.m2;
    TW *F = static_cast<TW *>(L.F), *V = static_cast<TW *>(L.V);
    TW *tf2 = sm, *tf1 = tf2 + 3 * g.m2;
    TW *S = sm + PersistSmem::b_tab(g.m1, g.m2);

    if (!g.c1) {
        // by rows: coarse row r = item * per + warp of the m0 x m1 rows
        const int r = item * per + warp;
        const bool mine = warp < per && r < g.m0 * g.m1;
        TW *row = S + warp * persist_round4(g.m2);
        if (mine) persist_stage<TW>(row, F + (int64_t)r * g.m2, g.m2, 1, lane);
        cp_async_commit();
        if (g.c2) persist_table<TW>(tf2, g.f2, 3 * g.m2);
        cp_async_wait<0>();
        __syncthreads();
        if (mine) {
            if (g.c2) persist_warp_solve<TW>(row, g.m2, tf2, lane);
            for (int x = lane; x < g.m2; x += 32) {
                const int64_t o = (int64_t)r * g.m2 + x;
                if constexpr (MODE == MODE_DEC) V[o] += row[x];
                else F[o] = row[x];
            }
        }
        return;
    }

    const int Z = item;
    TW *Fz = F + (int64_t)Z * mc;
    for (int64_t e = tid; e < mc; e += nt) cp_async_elem<TW>(S + e, Fz + e, true);
    cp_async_commit();
    if (g.c2) persist_table<TW>(tf2, g.f2, 3 * g.m2);
    persist_table<TW>(tf1, g.f1, 3 * g.m1);
    cp_async_wait<0>();
    __syncthreads();
    if (g.c2)
        for (int Yr = tid; Yr < g.m1; Yr += nt) persist_line_solve<TW>(S + (int64_t)Yr * g.m2, 1, g.m2, tf2);
    __syncthreads();
    for (int x = tid; x < g.m2; x += nt) persist_line_solve<TW>(S + x, g.m2, g.m1, tf1);
    __syncthreads();
    if constexpr (MODE == MODE_DEC) {
        TW *Vz = V + (int64_t)Z * mc;
        for (int64_t e = tid; e < mc; e += nt) Vz[e] += S[e];
    } else {
        for (int64_t e = tid; e < mc; e += nt) Fz[e] = S[e];
    }
}

// ---------------------------------------------------------------------------
// Phase D (recomposition): fine plane(s), U = C + Pi (V - z) on the nodes
// outside the coarse grid, V - z on the coarse nodes.
// ---------------------------------------------------------------------------

template <typename XT, typename TW>
__device__ __forceinline__ void persist_d_row(const PGeo<TW> &g, XT *xrow, const XT *rb, int i1, bool podd,
                                              const TW *tw1, const TW *tw2, const TW *c0, const TW *c1, int lane)
{
    const int q1 = g.c1 & i1 & 1;
    const bool even_row = !podd && !q1;
    const TW wl1 = q1 ? tw1[2 * i1] : TW(1), wr1 = q1 ? tw1[2 * i1 + 1] : TW(0);
    if (g.c2) {
        // lane takes the column pairs (2j, 2j+1), as in phase A
        const int np2 = (g.n2 + 1) >> 1;
        for (int j = lane; j < np2; j += 32) {
            const bool ho = 2 * j + 1 < g.n2;
            XT ue, uo = XT(0);
            if (ho) Pair2<XT>::load(rb, j, ue, uo);
            else ue = rb[2 * j];
            const TW a0 = c0[j], a1 = q1 ? c1[j] : a0;
            // even column: V - z on a coarse node, else C + the interpolant
            xrow[2 * j] = static_cast<XT>(even_row ? a0 : static_cast<TW>(ue) + (wl1 * a0 + wr1 * a1));
            if (ho) {
                TW wl2, wr2;
                Pair2<TW>::load(tw2, 2 * j + 1, wl2, wr2);
                const TW b0 = c0[j + 1], b1 = q1 ? c1[j + 1] : b0;
                const TW x0 = wl2 * a0 + wr2 * b0, x1 = wl2 * a1 + wr2 * b1;
                xrow[2 * j + 1] = static_cast<XT>(static_cast<TW>(uo) + (wl1 * x0 + wr1 * x1));
            }
        }
        return;
    }
    // P = I along dim 2
    for (int i2 = lane; i2 < g.n2; i2 += 32)
        xrow[i2] = static_cast<XT>(even_row ? c0[i2] : static_cast<TW>(rb[i2]) + (wl1 * c0[i2] + wr1 * c1[i2]));
}

template <typename XT, typename TW>
__device__ void persist_d(const PersistLevel &L, int item, int per, TW *sm)
{
    const PGeo<TW> g = pgeo<TW>(L);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t np = (int64_t)g.n1 * g.n2, mc = (int64_t)g.m1 * g.m2;
    const int rn = persist_round4(g.n2), rm = persist_round4(g.m2);
    XT *X = static_cast<XT *>(L.X);
    const TW *V = static_cast<const TW *>(L.V), *Zc = static_cast<const TW *>(L.F);
    TW *tw1 = sm, *tw2 = tw1 + 2 * g.n1;
    TW *wb = sm + PersistSmem::d_tab(g.n1, g.n2) + warp * PersistSmem::d_warp(g.c1, g.n2, g.m2);

    if (!g.c1) {
        // by rows; W = V - z of the coarse row(s) computed from the staged
        // rows of V and z
        const int r = item * per + warp;
        const bool mine = warp < per && r < g.n0 * g.n1;
        const int i0 = mine ? r / g.n1 : 0, i1 = mine ? r % g.n1 : 0;
        const bool podd = g.c0 && (i0 & 1);
        const int64_t ro = (int64_t)i0 * np + (int64_t)i1 * g.n2;
        XT *rb = reinterpret_cast<XT *>(wb);
        TW *sv = wb + rn;  // V, z of the coarse row (and the next coarse plane's when odd)
        if (mine) {
            persist_stage<XT>(rb, X + ro, g.n2, 1, lane);
            const int64_t o = (int64_t)(i0 >> g.c0) * mc + (int64_t)i1 * g.m2;
            persist_stage<TW>(sv, V + o, g.m2, 1, lane);
            persist_stage<TW>(sv + rm, Zc + o, g.m2, 1, lane);
            if (podd) {
                persist_stage<TW>(sv + 2 * rm, V + o + mc, g.m2, 1, lane);
                persist_stage<TW>(sv + 3 * rm, Zc + o + mc, g.m2, 1, lane);
            }
        }
        cp_async_commit();
        if (g.c2) persist_table<TW>(tw2, g.w2, 2 * g.n2);
        cp_async_wait<0>();
        __syncthreads();
        if (mine) {
            const TW wl = podd ? __ldg(g.w0 + 2 * i0) : TW(0), wr = podd ? __ldg(g.w0 + 2 * i0 + 1) : TW(0);
            // W in place of the first source row (each lane its own columns)
            for (int x = lane; x < g.m2; x += 32)
                sv[x] = podd ? wl * (sv[x] - sv[rm + x]) + wr * (sv[2 * rm + x] - sv[3 * rm + x]) : sv[x] - sv[rm + x];
            __syncwarp();
            persist_d_row<XT, TW>(g, X + ro, rb, i1, podd, tw1, tw2, sv, sv, lane);
        }
        return;
    }

    // a plane with an active dim 1: warp w takes the contiguous pairs
    // [w P, w P + P), so that the coarse row Y+1 of one pair is row Y of the
    // next; per pair the two fine rows and the sources of W row Y+1 are
    // staged one pair ahead
    const int i0 = item;
    const bool podd = g.c0 && (i0 & 1);
    const TW wl = podd ? __ldg(g.w0 + 2 * i0) : TW(0), wr = podd ? __ldg(g.w0 + 2 * i0 + 1) : TW(0);
    XT *Xp = X + (int64_t)i0 * np;
    const int64_t co = (int64_t)(i0 >> g.c0) * mc;
    TW *wA = wb, *wB = wb + rm;
    TW *sets = wb + 2 * rm;
    auto row = [&](int set, int k) { return reinterpret_cast<XT *>(sets + set * (2 * rn + 4 * rm) + k * rn); };
    auto srcs = [&](int set) { return sets + set * (2 * rn + 4 * rm) + 2 * rn; };
    auto stage_src = [&](int Y, int set) {  // V, z of coarse row Y (both planes when odd)
        TW *s = srcs(set);
        const int64_t o = co + (int64_t)Y * g.m2;
        persist_stage<TW>(s, V + o, g.m2, 1, lane);
        persist_stage<TW>(s + rm, Zc + o, g.m2, 1, lane);
        if (podd) {
            persist_stage<TW>(s + 2 * rm, V + o + mc, g.m2, 1, lane);
            persist_stage<TW>(s + 3 * rm, Zc + o + mc, g.m2, 1, lane);
        }
    };
    auto make_w = [&](int set, TW *w) {
        const TW *s = srcs(set);
        for (int x = lane; x < g.m2; x += 32)
            w[x] = podd ? wl * (s[x] - s[rm + x]) + wr * (s[2 * rm + x] - s[3 * rm + x]) : s[x] - s[rm + x];
    };
    auto stage_pair = [&](int Y, int set) {
        persist_stage<XT>(row(set, 0), Xp + (int64_t)(2 * Y) * g.n2, g.n2, 1, lane);
        if (2 * Y + 1 < g.n1) {
            persist_stage<XT>(row(set, 1), Xp + (int64_t)(2 * Y + 1) * g.n2, g.n2, 1, lane);
            stage_src(Y + 1, set);
        }
    };
    const int P = (g.m1 + kPersistWarps - 1) / kPersistWarps;
    const int Yb = warp * P, Ye = min(g.m1, Yb + P);
    if (Yb < Ye) {
        stage_src(Yb, 0);
        cp_async_commit();
    }
    persist_table<TW>(tw1, g.w1, 2 * g.n1);
    if (g.c2) persist_table<TW>(tw2, g.w2, 2 * g.n2);
    __syncthreads();  // the tables
    if (Yb >= Ye) return;
    cp_async_wait<0>();
    __syncwarp();
    make_w(0, wA);
    __syncwarp();
    stage_pair(Yb, 0);
    cp_async_commit();
    for (int Y = Yb, set = 0; Y < Ye; ++Y, set ^= 1) {
        if (Y + 1 < Ye) stage_pair(Y + 1, set ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const bool two = 2 * Y + 1 < g.n1;
        if (two) make_w(set, wB);
        __syncwarp();
        persist_d_row<XT, TW>(g, Xp + (int64_t)(2 * Y) * g.n2, row(set, 0), 2 * Y, podd, tw1, tw2, wA, wA, lane);
        if (two)
            persist_d_row<XT, TW>(g, Xp + (int64_t)(2 * Y + 1) * g.n2, row(set, 1), 2 * Y + 1, podd, tw1, tw2, wA,
                                  wB, lane);
        __syncwarp();
        TW *t = wA;
        wA = wB;
        wB = t;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Final placement (decomposition): the final value at a coarse node of grid
// level i is that of V_i as the deeper levels left it (their coefficient
// where the node is outside their coarse grid, else recursively theirs; the
// last grid level's V holds its final values).  Coarse rows (Z, Y) of one
// level, two per warp, lanes along the row.
// ---------------------------------------------------------------------------
template <typename TX, typename TW>
__device__ void persist_place(const PersistParams &p, const PersistTask &t, int item)
{
    const PersistLevel *lv = p.lv + t.level;
    const PersistLevel &L = lv[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m1 = L.m[1], m2 = L.m[2], n1 = L.n[1], n2 = L.n[2];
    const int rows = L.m[0] * m1;
    constexpr int U = 4;
    for (int rr = 0; rr < kPersistPlaceRows / kPersistWarps; ++rr) {
        const int r = item * kPersistPlaceRows + rr * kPersistWarps + warp;
        if (r >= rows) break;
        const int Z = r / m1, Y = r % m1;
        const int64_t orow = ((int64_t)(Z << L.co[0]) * n1 + (Y << L.co[1])) * n2;
        for (int x0 = lane; x0 < m2; x0 += 32 * U) {
            const TW *src[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int xc = x0 + 32 * u;
                src[u] = nullptr;
                if (xc >= m2) continue;
                int k = 0, z = Z, y = Y, x = xc;
                while (k + 1 < t.nlevels) {
                    const PersistLevel &N = lv[k + 1];
                    const int odd = (N.co[0] & z) | (N.co[1] & y) | (N.co[2] & x);
                    if (odd & 1) break;
                    z >>= N.co[0];
                    y >>= N.co[1];
                    x >>= N.co[2];
                    ++k;
                }
                const PersistLevel &K = lv[k];
                src[u] = static_cast<const TW *>(K.V) + ((int64_t)z * K.m[1] + y) * K.m[2] + x;
            }
            TW v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (src[u]) v[u] = *src[u];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (src[u]) {
                    const int64_t o = orow + ((x0 + 32 * u) << L.co[2]);
                    if (L.first) static_cast<TX *>(L.X)[o] = static_cast<TX>(v[u]);
                    else static_cast<TW *>(L.X)[o] = v[u];
                }
        }
    }
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------

// Global nanosecond timer (measurement only).
__device__ __forceinline__ unsigned long long persist_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Thread 0: wait, bounded, until `need` items of a task are done.
__device__ __forceinline__ void persist_wait(const PersistParams &p, const unsigned *cnt, unsigned need)
{
    int spins = 0;
    while (persist_ld_acquire(cnt) < need && spins < p.spin_limit) {
        __nanosleep(64);
        ++spins;
    }
    if (persist_ld_acquire(cnt) < need) atomicOr(p.status, 1u);
}

template <typename TX, typename TW, int MODE>
__global__ void __launch_bounds__(kPersistThreads, sizeof(TW) == 4 ? 2 : 1) k_persist(PersistParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ int2 s_e;
    __shared__ PersistTask s_t;
    __shared__ unsigned long long s_t1;
    TW *sm = reinterpret_cast<TW *>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = (int)atomicAdd(p.next, 1u);
            s_item = it;
            if (it < p.nitems) {
                const int2 e = p.items[it];
                const PersistTask t = p.tasks[e.x];
                const unsigned long long t0 = p.prof ? persist_clock() : 0ull;
                for (int d = 0; d < 2; ++d)
                    if (t.dep[d] >= 0) persist_wait(p, p.done + t.dep[d], (unsigned)p.tasks[t.dep[d]].nitems);
                if (p.stall && it == 0) persist_wait(p, p.zero, 1u);  // a count nothing reaches
                __threadfence();
                s_e = e;
                s_t = t;
                if (p.prof) {
                    s_t1 = persist_clock();
                    atomicAdd(p.prof + kPersistKinds + t.kind, s_t1 - t0);
                }
            }
        }
        __syncthreads();
        if (s_item >= p.nitems) break;
        const int2 e = s_e;
        const PersistTask t = s_t;
        switch (t.kind) {
        case PK_A: {
            const PersistLevel &L = p.lv[t.level];
            if constexpr (sizeof(TX) == sizeof(TW)) {
                persist_a<TW, TW, MODE>(L, e.y, t.per, sm);
            } else {
                if (L.first) persist_a<TX, TW, MODE>(L, e.y, t.per, sm);
                else persist_a<TW, TW, MODE>(L, e.y, t.per, sm);
            }
            break;
        }
        case PK_B: persist_b<TW, MODE>(p.lv[t.level], e.y, t.per, sm); break;
        case PK_C: persist_c<TW>(p.lv[t.level], e.y, sm); break;
        case PK_D:
            if constexpr (MODE == MODE_REC) {
                const PersistLevel &L = p.lv[t.level];
                if constexpr (sizeof(TX) == sizeof(TW)) {
                    persist_d<TW, TW>(L, e.y, t.per, sm);
                } else {
                    if (L.first) persist_d<TX, TW>(L, e.y, t.per, sm);
                    else persist_d<TW, TW>(L, e.y, t.per, sm);
                }
            }
            break;
        case PK_SMALL: small_run<TW, TW, MODE>(p.small[t.level], smem_raw); break;
        case PK_PLACE:
            if constexpr (MODE == MODE_DEC) persist_place<TX, TW>(p, t, e.y);
            break;
        default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p.done + e.x) : "memory");
            if (p.prof) {
                atomicAdd(p.prof + t.kind, persist_clock() - s_t1);
                atomicAdd(p.prof + 2 * kPersistKinds + t.kind, 1ull);
            }
        }
    }
}

}  // namespace mg
