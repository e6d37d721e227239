// multi.cuh -- the coarse end of the hierarchy in one cooperative launch.
//
// Below some size a level is too small to fill the GPU and its dozen
// dependent launches cost more than its work.  k_multi runs the levels whose
// arrays have sides <= 129 nodes with every block of the grid, phase after
// phase, separated by a grid barrier; each block takes whole planes or lines
// of a level and stages them in shared memory.  The steps are those of the
// tiled path (Section II-A, Eq. 1-2; Section III-A):
//   A  per fine plane i0: coefficients C = U - Pi U_coarse (decomposition;
//      written back in place), the gather of the coarse nodes into V, and
//      the load vector reduced along dims 2 and 1 (G = K_1 (x) K_2 C);
//   B  per coarse plane Z: F = K_0 G, then M_{l-1} z = F along dims 2 and 1;
//   C  per coarse row Y: the solve along dim 0, then V += z (decomposition)
//      or z kept in F (recomposition);
//   D  (recomposition) per fine plane: U = C + Pi (V - z), coarse nodes V - z.
// Decomposition: A, B, C per level, finest first; block 0 then runs the
// remaining levels in shared memory (small.cuh); one last phase places each
// level's final coarse values into its array.  Recomposition: the load
// vectors and corrections of all levels first (they depend only on stored
// coefficients; phase t runs A of level t, B of level t-1 and C of level
// t-2 together, block 0 the shared-memory levels in phase nd), then D per
// level, coarsest first.
//
// The barrier needs every block resident: the kernel is launched as a
// cooperative launch.  Its wait is bounded; a wait that runs out (which a
// co-resident grid does not cause) sets the third barrier word and the block
// goes on.
#pragma once

#include "common.cuh"
#include "multi_params.h"
#include "params.h"
#include "small.cuh"

namespace mg {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: bar[0] counts arrivals, bar[1] is the generation, bar[2]
// records a wait that ran out.  The block's writes are ordered before
// thread 0's release arrival by the block barrier; the last arrival resets
// the count and releases the next generation, which the others acquire.
__device__ __forceinline__ void multi_barrier(unsigned *bar, int limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_gpu(bar + 1);
        unsigned prev;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(prev) : "l"(bar) : "memory");
        if (prev + 1 == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
        } else {
            int it = 0;
            while (ld_acquire_gpu(bar + 1) == g && it < limit) {
                __nanosleep(20);
                ++it;
            }
            if (ld_acquire_gpu(bar + 1) == g) atomicOr(bar + 2, 1u);
        }
    }
    __syncthreads();
}

template <typename TW>
struct MGeo {
    int n0, n1, n2, m0, m1, m2;
    int a0, a1, a2;           // 1 for an active dimension
    const TW *w0, *w1, *w2, *k0, *k1, *k2, *f0, *f1, *f2;
};

template <typename TW>
__device__ __forceinline__ MGeo<TW> mgeo(const MultiLevel &L)
{
    MGeo<TW> g;
    g.n0 = L.n[0]; g.n1 = L.n[1]; g.n2 = L.n[2];
    g.m0 = L.m[0]; g.m1 = L.m[1]; g.m2 = L.m[2];
    g.a0 = g.n0 > 1; g.a1 = g.n1 > 1; g.a2 = g.n2 > 1;
    g.w0 = static_cast<const TW *>(L.w[0]); g.w1 = static_cast<const TW *>(L.w[1]);
    g.w2 = static_cast<const TW *>(L.w[2]);
    g.k0 = static_cast<const TW *>(L.k[0]); g.k1 = static_cast<const TW *>(L.k[1]);
    g.k2 = static_cast<const TW *>(L.k[2]);
    g.f0 = static_cast<const TW *>(L.fac[0]); g.f1 = static_cast<const TW *>(L.fac[1]);
    g.f2 = static_cast<const TW *>(L.fac[2]);
    return g;
}

// Asynchronous copy of n elements from global into shared memory (one copy
// per element, all in flight); the caller commits, waits and synchronizes.
template <typename TW>
__device__ __forceinline__ void multi_copy_async(TW *dst, const TW *src, int n)
{
    for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async_elem<TW>(dst + e, src + e, true);
}

// n elements of the level array into shared memory: asynchronous copies
// when the types are equal (committed with any copies issued before), else
// (FP32 array, FP64 arithmetic) four per thread at a time through
// registers.  The caller synchronizes the block before reading dst.
template <typename XT, typename TW>
__device__ __forceinline__ void multi_stage(TW *dst, const XT *src, int n)
{
    if constexpr (sizeof(XT) == sizeof(TW)) {
        multi_copy_async<TW>(dst, reinterpret_cast<const TW *>(src), n);
        cp_async_commit();
        cp_async_wait<0>();
    } else {
        cp_async_commit();
        constexpr int B = 4;
        const int nt = blockDim.x;
        for (int e0 = threadIdx.x; e0 < n; e0 += B * nt) {
            XT v[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < n) v[u] = src[e];
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < n) dst[e] = static_cast<TW>(v[u]);
            }
        }
        cp_async_wait<0>();
    }
}

// Phase A on fine plane i0.  Shared memory: the tables (w1, w2: two weights
// per fine node; k1, k2: five stencil entries per coarse node), the plane P
// (n1 x n2), then W: first the plane's coarse grid (decomposition of an odd
// plane: the dim-0 interpolation of its neighbours' coarse nodes), then
// H = K_2 C (n1 x m2).  Rows go to warps, columns to lanes.
template <typename XT, typename TW, int MODE>
__device__ void multi_phase_a(const MultiLevel &L, int i0, TW *sm)
{
    const MGeo<TW> g = mgeo<TW>(L);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int np = g.n1 * g.n2, mc = g.m1 * g.m2;
    TW *tw1 = sm, *tw2 = tw1 + 2 * g.n1, *tk1 = tw2 + 2 * g.n2, *tk2 = tk1 + 5 * g.m1;
    TW *P = sm + kMultiTabElems, *W = P + np;
    XT *Xp = static_cast<XT *>(L.X) + (int64_t)i0 * np;
    const bool podd = g.a0 && (i0 & 1);
    if (g.a1) {
        multi_copy_async<TW>(tw1, g.w1, 2 * g.n1);
        multi_copy_async<TW>(tk1, g.k1, 5 * g.m1);
    }
    if (g.a2) {
        multi_copy_async<TW>(tw2, g.w2, 2 * g.n2);
        multi_copy_async<TW>(tk2, g.k2, 5 * g.m2);
    }
    multi_stage<XT, TW>(P, Xp, np);
    if (MODE == MODE_DEC && podd) {
        const TW wl = __ldg(g.w0 + 2 * i0), wr = __ldg(g.w0 + 2 * i0 + 1);
        const XT *xa = Xp - np, *xb = Xp + np;
        for (int Y = warp; Y < g.m1; Y += nw) {
            const int ro = (g.a1 ? 2 * Y : 0) * g.n2;
            constexpr int B = 3;
            XT va[B], vb[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int Xc = lane + 32 * u;
                if (Xc < g.m2) {
                    va[u] = xa[ro + (g.a2 ? 2 * Xc : 0)];
                    vb[u] = xb[ro + (g.a2 ? 2 * Xc : 0)];
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int Xc = lane + 32 * u;
                if (Xc < g.m2) W[Y * g.m2 + Xc] = wl * static_cast<TW>(va[u]) + wr * static_cast<TW>(vb[u]);
            }
        }
    }
    __syncthreads();
    if (!podd) {  // coarse grid of the plane, gathered into V
        TW *V = static_cast<TW *>(L.V) + (int64_t)(i0 >> 1) * mc;
        for (int Y = warp; Y < g.m1; Y += nw) {
            const TW *prow = P + (g.a1 ? 2 * Y : 0) * g.n2;
            for (int Xc = lane; Xc < g.m2; Xc += 32) {
                const TW v = prow[g.a2 ? 2 * Xc : 0];
                W[Y * g.m2 + Xc] = v;
                V[Y * g.m2 + Xc] = v;
            }
        }
        __syncthreads();
    }
    if constexpr (MODE == MODE_DEC) {
        for (int i1 = warp; i1 < g.n1; i1 += nw) {
            const int q1 = g.a1 & i1 & 1;
            const TW wl1 = q1 ? tw1[2 * i1] : TW(1), wr1 = q1 ? tw1[2 * i1 + 1] : TW(0);
            const TW *c0 = W + (i1 >> 1) * g.m2, *c1 = c0 + q1 * g.m2;
            TW *prow = P + i1 * g.n2;
            XT *xrow = Xp + i1 * g.n2;
            const bool even_row = !podd && !q1;
            TW I[kMultiRowChunks], u[kMultiRowChunks];
#pragma unroll
            for (int k = 0; k < kMultiRowChunks; ++k) {  // every load of the row first
                const int i2 = lane + 32 * k;
                const int q2 = g.a2 & i2 & 1, x = i2 >> 1;
                if (i2 < g.n2) {
                    const TW wl2 = q2 ? tw2[2 * i2] : TW(1), wr2 = q2 ? tw2[2 * i2 + 1] : TW(0);
                    const TW x0 = wl2 * c0[x] + wr2 * c0[x + q2];
                    const TW x1 = wl2 * c1[x] + wr2 * c1[x + q2];
                    I[k] = wl1 * x0 + wr1 * x1;
                    u[k] = prow[i2];
                }
            }
#pragma unroll
            for (int k = 0; k < kMultiRowChunks; ++k) {
                const int i2 = lane + 32 * k;
                const int q2 = g.a2 & i2 & 1;
                if (i2 < g.n2 && !(even_row && !q2)) {  // not a coarse node
                    const XT c = static_cast<XT>(u[k] - I[k]);
                    xrow[i2] = c;
                    prow[i2] = static_cast<TW>(c);  // the load vector sees the stored value
                }
            }
        }
        __syncthreads();
    }
    // H(i1, X) = sum_c K_2[X][c] C(i1, 2X - 2 + c), C = 0 on coarse nodes
    for (int i1 = warp; i1 < g.n1; i1 += nw) {
        const bool rodd = podd || (g.a1 & i1 & 1);
        const TW *row = P + i1 * g.n2;
        TW h[kMultiCoarseChunks];
#pragma unroll
        for (int k = 0; k < kMultiCoarseChunks; ++k) {
            const int Xc = lane + 32 * k;
            h[k] = TW(0);
            if (Xc < g.m2) {
                if (g.a2) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) {
                        const int i2 = 2 * Xc - 2 + c;
                        if (i2 >= 0 && i2 < g.n2 && (rodd || (c & 1))) h[k] += tk2[5 * Xc + c] * row[i2];
                    }
                } else if (rodd) {
                    h[k] = row[0];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kMultiCoarseChunks; ++k) {
            const int Xc = lane + 32 * k;
            if (Xc < g.m2) W[i1 * g.m2 + Xc] = h[k];
        }
    }
    __syncthreads();
    // G(i0, Y, X) = sum_b K_1[Y][b] H(2Y - 2 + b, X)
    TW *G = static_cast<TW *>(L.G) + (int64_t)i0 * mc;
    for (int Y = warp; Y < g.m1; Y += nw) {
        TW k[5];
        int r[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int i1 = 2 * Y - 2 + b;
            const bool ok = g.a1 ? (i1 >= 0 && i1 < g.n1) : (b == 2);
            k[b] = ok ? (g.a1 ? tk1[5 * Y + b] : TW(1)) : TW(0);
            r[b] = ok ? (g.a1 ? i1 : 0) : 0;
        }
        TW v[kMultiCoarseChunks];
#pragma unroll
        for (int c = 0; c < kMultiCoarseChunks; ++c) {
            const int Xc = lane + 32 * c;
            v[c] = TW(0);
            if (Xc < g.m2) {
#pragma unroll
                for (int b = 0; b < 5; ++b) v[c] += k[b] * W[r[b] * g.m2 + Xc];
            }
        }
#pragma unroll
        for (int c = 0; c < kMultiCoarseChunks; ++c) {
            const int Xc = lane + 32 * c;
            if (Xc < g.m2) G[Y * g.m2 + Xc] = v[c];
        }
    }
    __syncthreads();
}

// Phase B on coarse plane Z: the G planes 2Z-2 .. 2Z+2 and the LU factors of
// dims 2 and 1 staged in shared memory, F = K_0 G (into the first slot), the
// solves along dims 2 and 1 (one thread per line), the plane back to F.
template <typename TW>
__device__ void multi_phase_b(const MultiLevel &L, int Z, TW *sm)
{
    const MGeo<TW> g = mgeo<TW>(L);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mc = g.m1 * g.m2;
    const TW *G = static_cast<const TW *>(L.G);
    TW *tf2 = sm, *tf1 = tf2 + 3 * g.m2;
    TW *S = sm + kMultiTabElems;
    const int lo = g.a0 ? max(0, 2 * Z - 2) : 0, hi = g.a0 ? min(g.n0 - 1, 2 * Z + 2) : 0;
    if (g.a2) multi_copy_async<TW>(tf2, g.f2, 3 * g.m2);
    if (g.a1) multi_copy_async<TW>(tf1, g.f1, 3 * g.m1);
    multi_stage<TW, TW>(S, G + (int64_t)lo * mc, (hi - lo + 1) * mc);
    __syncthreads();
    if (g.a0) {
        TW k[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) k[a] = __ldg(g.k0 + 5 * Z + a);
        for (int e = tid; e < mc; e += nt) {
            TW f = TW(0);
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const int i0 = 2 * Z - 2 + a;
                if (i0 >= lo && i0 <= hi) f += k[a] * S[(i0 - lo) * mc + e];
            }
            S[e] = f;  // slot 0: read above by this thread only
        }
    }
    __syncthreads();
    if (g.a2)
        for (int Y = tid; Y < g.m1; Y += nt) line_solve_smem<TW>(S + Y * g.m2, 1, g.m2, tf2);
    __syncthreads();
    if (g.a1)
        for (int Xc = tid; Xc < g.m2; Xc += nt) line_solve_smem<TW>(S + Xc, g.m2, g.m1, tf1);
    __syncthreads();
    TW *F = static_cast<TW *>(L.F) + (int64_t)Z * mc;
    for (int e = tid; e < mc; e += nt) F[e] = S[e];
    __syncthreads();
}

// Phase C on coarse row Y: the lines along dim 0 (an m0 x m2 slice), then
// V += z (decomposition) or z back into F (recomposition).  Shared memory:
// the LU factors of dim 0, the slice of F, then (decomposition) that of V.
template <typename TW, int MODE>
__device__ void multi_phase_c(const MultiLevel &L, int Y, TW *sm)
{
    const MGeo<TW> g = mgeo<TW>(L);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    TW *F = static_cast<TW *>(L.F), *V = static_cast<TW *>(L.V);
    if (!g.a0) {  // 2D: z is complete after phase B
        if constexpr (MODE == MODE_DEC)
            for (int Xc = tid; Xc < g.m2; Xc += nt) V[Y * g.m2 + Xc] += F[Y * g.m2 + Xc];
        return;
    }
    const int ns = g.m0 * g.m2, rs = g.m1 * g.m2;
    TW *tf0 = sm, *S = sm + kMultiTabElems, *S2 = S + ns;
    multi_copy_async<TW>(tf0, g.f0, 3 * g.m0);
    for (int Z = warp; Z < g.m0; Z += nw) {
        const int64_t o = (int64_t)Z * rs + Y * g.m2;
        for (int Xc = lane; Xc < g.m2; Xc += 32) {
            cp_async_elem<TW>(S + Z * g.m2 + Xc, F + o + Xc, true);
            if (MODE == MODE_DEC) cp_async_elem<TW>(S2 + Z * g.m2 + Xc, V + o + Xc, true);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int Xc = tid; Xc < g.m2; Xc += nt) line_solve_smem<TW>(S + Xc, g.m2, g.m0, tf0);
    __syncthreads();
    for (int Z = warp; Z < g.m0; Z += nw) {
        const int64_t o = (int64_t)Z * rs + Y * g.m2;
        for (int Xc = lane; Xc < g.m2; Xc += 32) {
            if constexpr (MODE == MODE_DEC) V[o + Xc] = S2[Z * g.m2 + Xc] + S[Z * g.m2 + Xc];
            else F[o + Xc] = S[Z * g.m2 + Xc];
        }
    }
    __syncthreads();
}

// Phase D (recomposition) on fine plane i0: the coarse grid V - z of the
// plane (odd plane: interpolated along dim 0) into W, then every node.
template <typename XT, typename TW>
__device__ void multi_phase_d(const MultiLevel &L, int i0, TW *sm)
{
    const MGeo<TW> g = mgeo<TW>(L);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int np = g.n1 * g.n2, mc = g.m1 * g.m2;
    TW *tw1 = sm, *tw2 = tw1 + 2 * g.n1;
    TW *P = sm + kMultiTabElems, *W = P + np;
    XT *Xp = static_cast<XT *>(L.X) + (int64_t)i0 * np;
    const bool podd = g.a0 && (i0 & 1);
    const TW *V = static_cast<const TW *>(L.V) + (int64_t)(i0 >> 1) * mc;
    const TW *Z = static_cast<const TW *>(L.F) + (int64_t)(i0 >> 1) * mc;
    if (g.a1) multi_copy_async<TW>(tw1, g.w1, 2 * g.n1);
    if (g.a2) multi_copy_async<TW>(tw2, g.w2, 2 * g.n2);
    multi_stage<XT, TW>(P, Xp, np);
    constexpr int B = 4;
    if (podd) {
        const TW wl = __ldg(g.w0 + 2 * i0), wr = __ldg(g.w0 + 2 * i0 + 1);
        for (int e0 = tid; e0 < mc; e0 += B * nt) {
            TW v[B][4];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < mc) {
                    v[u][0] = V[e];
                    v[u][1] = Z[e];
                    v[u][2] = V[mc + e];
                    v[u][3] = Z[mc + e];
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < mc) W[e] = wl * (v[u][0] - v[u][1]) + wr * (v[u][2] - v[u][3]);
            }
        }
    } else {
        for (int e0 = tid; e0 < mc; e0 += B * nt) {
            TW v[B][2];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < mc) {
                    v[u][0] = V[e];
                    v[u][1] = Z[e];
                }
            }
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int e = e0 + u * nt;
                if (e < mc) W[e] = v[u][0] - v[u][1];
            }
        }
    }
    __syncthreads();
    for (int i1 = warp; i1 < g.n1; i1 += nw) {
        const int q1 = g.a1 & i1 & 1;
        const TW wl1 = q1 ? tw1[2 * i1] : TW(1), wr1 = q1 ? tw1[2 * i1 + 1] : TW(0);
        const TW *c0 = W + (i1 >> 1) * g.m2, *c1 = c0 + q1 * g.m2;
        const TW *prow = P + i1 * g.n2;
        XT *xrow = Xp + i1 * g.n2;
        const bool even_row = !podd && !q1;
        TW r[kMultiRowChunks];
#pragma unroll
        for (int k = 0; k < kMultiRowChunks; ++k) {
            const int i2 = lane + 32 * k;
            const int q2 = g.a2 & i2 & 1, x = i2 >> 1;
            if (i2 < g.n2) {
                if (even_row && !q2) {
                    r[k] = c0[x];  // coarse node: V - z
                } else {
                    const TW wl2 = q2 ? tw2[2 * i2] : TW(1), wr2 = q2 ? tw2[2 * i2 + 1] : TW(0);
                    const TW x0 = wl2 * c0[x] + wr2 * c0[x + q2];
                    const TW x1 = wl2 * c1[x] + wr2 * c1[x + q2];
                    r[k] = prow[i2] + (wl1 * x0 + wr1 * x1);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kMultiRowChunks; ++k) {
            const int i2 = lane + 32 * k;
            if (i2 < g.n2) xrow[i2] = static_cast<XT>(r[k]);
        }
    }
    __syncthreads();
}

// Final coarse values of every decomposed grid level into its array.  The
// final value at a coarse node of level i is that of V_i, which the next
// level transformed in place: its coefficient where the node is not coarse
// there, else (recursively) the next level's final value; the last V holds
// its final values.  Reads only nodes that this phase does not write.
template <typename TX, typename TW>
__device__ void multi_place_all(const MultiParams &p)
{
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x), gs = (int)(gridDim.x * blockDim.x);
    for (int i = 0; i < p.nd; ++i) {
        const MultiLevel &L = p.lv[i];
        const int n1 = L.n[1], n2 = L.n[2], m1 = L.m[1], m2 = L.m[2];
        const int a0 = L.n[0] > 1, a1 = n1 > 1, a2 = n2 > 1;
        const int tot = L.m[0] * m1 * m2;
        for (int e = gtid; e < tot; e += gs) {
            const int Xc = e % m2, r = e / m2;
            const int Y = r % m1, Z = r / m1;
            int k = i, z = Z, y = Y, x = Xc;
            while (k + 1 < p.nd) {
                const MultiLevel &N = p.lv[k + 1];
                const int odd = ((N.n[0] > 1) & z) | ((N.n[1] > 1) & y) | ((N.n[2] > 1) & x);
                if (odd & 1) break;
                z >>= 1;
                y >>= 1;
                x >>= 1;
                ++k;
            }
            const MultiLevel &K = p.lv[k];
            const TW v = static_cast<const TW *>(K.V)[((int64_t)z * K.m[1] + y) * K.m[2] + x];
            const int64_t o = ((int64_t)(a0 ? 2 * Z : 0) * n1 + (a1 ? 2 * Y : 0)) * n2 + (a2 ? 2 * Xc : 0);
            if (i == 0) static_cast<TX *>(L.X)[o] = static_cast<TX>(v);
            else static_cast<TW *>(L.X)[o] = v;
        }
    }
}

template <typename TX, typename TW, int MODE>
__device__ __forceinline__ void multi_a(const MultiParams &p, int i, int it, TW *sm)
{
    if (i == 0) multi_phase_a<TX, TW, MODE>(p.lv[0], it, sm);
    else multi_phase_a<TW, TW, MODE>(p.lv[i], it, sm);
}

template <typename TX, typename TW, int MODE>
__global__ void __launch_bounds__(kMultiThreads, 1) k_multi(MultiParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *sm = reinterpret_cast<TW *>(smem_raw);
    if constexpr (MODE == MODE_DEC) {
        for (int i = 0; i < p.nd; ++i) {
            const MultiLevel &L = p.lv[i];
            for (int it = blockIdx.x; it < L.n[0]; it += gridDim.x) multi_a<TX, TW, MODE_DEC>(p, i, it, sm);
            multi_barrier(p.bar, p.spin_limit);
            for (int it = blockIdx.x; it < L.m[0]; it += gridDim.x) multi_phase_b<TW>(L, it, sm);
            multi_barrier(p.bar, p.spin_limit);
            for (int it = blockIdx.x; it < L.m[1]; it += gridDim.x) multi_phase_c<TW, MODE_DEC>(L, it, sm);
            multi_barrier(p.bar, p.spin_limit);
        }
        if (p.small) {
            if (blockIdx.x == 0) small_run<TW, TW, MODE_DEC>(p.sp, smem_raw);
            multi_barrier(p.bar, p.spin_limit);
        }
        multi_place_all<TX, TW>(p);
    } else {
        // phase t: A of level t, B of level t-1, C of level t-2 (block 0 runs
        // the shared-memory levels in phase nd, after the last gather)
        for (int t = 0; t <= p.nd + 1; ++t) {
            const bool small_here = p.small && t == p.nd;
            const int b0 = small_here ? 1 : 0;
            if (small_here && blockIdx.x == 0) {
                small_run<TW, TW, MODE_REC>(p.sp, smem_raw);
            } else {
                const int na = (t < p.nd) ? p.lv[t].n[0] : 0;
                const int nb = (t >= 1 && t - 1 < p.nd) ? p.lv[t - 1].m[0] : 0;
                const int nc = (t >= 2) ? p.lv[t - 2].m[1] : 0;
                for (int it = (int)blockIdx.x - b0; it < na + nb + nc; it += (int)gridDim.x - b0) {
                    if (it < na) multi_a<TX, TW, MODE_REC>(p, t, it, sm);
                    else if (it < na + nb) multi_phase_b<TW>(p.lv[t - 1], it - na, sm);
                    else multi_phase_c<TW, MODE_REC>(p.lv[t - 2], it - na - nb, sm);
                }
            }
            multi_barrier(p.bar, p.spin_limit);
        }
        for (int i = p.nd - 1; i >= 0; --i) {
            const MultiLevel &L = p.lv[i];
            for (int it = blockIdx.x; it < L.n[0]; it += gridDim.x) {
                if (i == 0) multi_phase_d<TX, TW>(L, it, sm);
                else multi_phase_d<TW, TW>(L, it, sm);
            }
            if (i > 0) multi_barrier(p.bar, p.spin_limit);
        }
    }
}

}  // namespace mg
