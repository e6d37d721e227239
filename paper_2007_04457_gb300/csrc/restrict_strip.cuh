// restrict_strip.cuh -- load vector and coarse gather of one level, one warp
// per strip (both directions; same result as k_restrict up to rounding).
//
// Computes, like k_restrict (Section III-A-2),
//   F = (K_0 (x) K_1 (x) K_2) C,  C = A on N_l \ N_{l-1}, 0 on N_{l-1}
//   V = A restricted to N_{l-1}
// with a layout that needs no shared memory and no block barrier: a warp
// item is a strip of 30 coarse columns x TY coarse rows x a chunk of coarse
// planes.  Lane L covers coarse column X0 - 1 + L; lanes 1..30 compute, and
// lanes 0 and 31 only supply the neighbouring fine columns.  The warp streams
// the fine planes of its chunk; in every plane it loads the 2 TY + 3 fine
// rows that feed its coarse rows, two fine columns per lane (2X, 2X+1; the
// neighbours' values by shuffles), applies the dim-2 stencil per row and
// accumulates the dim-1 stencil into TY registers; the dim-0 stencil goes
// into rolling register accumulators over the plane pairs (odd plane 2Z-1,
// even plane 2Z).  Whether a fine row holds coarse nodes is a compile-time
// fact of the unrolled row loop, so coarse rows take the 2-tap form of the
// stencil.
//
// A strip or row block that would pass the last coarse column or row is
// shifted back to end there; its lanes or rows that another item owns
// compute but do not write.  Needs m2 >= 30 and m1 >= TY; smaller levels use
// k_restrict.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kStripThreads = 256;
constexpr int kStripCols = 30;  // coarse columns a warp computes

template <typename T>
struct StripRows {
    static constexpr int value = sizeof(T) == 4 ? 8 : 4;  // coarse rows per strip
};

// Fine columns lo, lo + 1 of a row (0 outside the grid or for an invalid
// row; INT: both inside).  Two scalar loads: measured faster here than one
// paired load.
template <typename T, bool INT>
__device__ __forceinline__ void strip_load2(const T *row, int lo, int n2, bool yok, T &a, T &b)
{
    if (INT) {
        a = row[lo];
        b = row[lo + 1];
    } else {
        a = (yok && lo >= 0 && lo < n2) ? row[lo] : T(0);
        b = (yok && lo + 1 >= 0 && lo + 1 < n2) ? row[lo + 1] : T(0);
    }
}

// The dim-2 and dim-1 restriction of fine plane z into g[0..TY): ODD = the
// plane index is odd (every node of it is a coefficient node).  Gathers the
// coarse values of owned nodes into V when `gather`.  FAST: every coarse row
// of the strip has the dim-1 stencil ku (kept in registers) and every row
// and column the strip reads lies inside the grid; else the rows are read
// from the table k1 and every load is checked.  Each lane reads the pair (2X, 2X+1) of a row
// whose plane and row indices have an even sum, else (2X-1, 2X) (these are
// the pairs that start on a two-element boundary, since n1 n2 and n2 are
// odd); the other three values of its five come from the neighbour lanes.
template <typename T, typename TW, int TY, bool ODD, bool FAST>
__device__ __forceinline__ void strip_plane(const T *__restrict__ plane, int n1, int n2, int Y0, int cx,
                                            const T (&kx)[5], const T (&ku)[5], const T *__restrict__ k1,
                                            T (&g)[TY], bool gather, TW *__restrict__ vplane, int yown, int m2,
                                            int X, bool xown)
{
#pragma unroll
    for (int j = 0; j < TY; ++j) g[j] = T(0);
    constexpr int R = 2 * TY + 3;
    T a[R], b[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {  // every load of the plane first
        const int y = 2 * Y0 - 2 + r;
        const bool yok = FAST || (y >= 0 && y < n1);
        const T *row = plane + (int64_t)(yok ? y : 0) * n2;
        const bool aligned = ((ODD ? 1 : 0) + r) % 2 == 0;  // fine row y has the parity of r
        strip_load2<T, FAST>(row, aligned ? cx : cx - 1, n2, yok, a[r], b[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool aligned = ((ODD ? 1 : 0) + r) % 2 == 0;
        // the five fine columns 2X-2 .. 2X+2 of row r
        T c0r, c1r, cm1, cm2, cp2;
        if (aligned) {  // a = col 2X, b = col 2X+1
            c0r = a[r];
            c1r = b[r];
            cm2 = __shfl_up_sync(0xffffffffu, a[r], 1);
            cm1 = __shfl_up_sync(0xffffffffu, b[r], 1);
            cp2 = __shfl_down_sync(0xffffffffu, a[r], 1);
        } else {  // a = col 2X-1, b = col 2X
            cm1 = a[r];
            c0r = b[r];
            c1r = __shfl_down_sync(0xffffffffu, a[r], 1);
            cp2 = __shfl_down_sync(0xffffffffu, b[r], 1);
            cm2 = __shfl_up_sync(0xffffffffu, b[r], 1);
        }
        const bool rodd = ODD || (r & 1);  // fine row 2 Y0 - 2 + r has the parity of r
        if (!ODD && !(r & 1) && gather) {
            // coarse values of the owned coarse rows
            const int Yr = Y0 - 1 + r / 2;
            if (Yr >= yown && Yr < Y0 + TY && xown) vplane[(int64_t)Yr * m2 + X] = static_cast<TW>(c0r);
        }
        T h;
        if (rodd) {
            h = fma_rn(kx[0], cm2, mul_rn(kx[1], cm1));
            h = fma_rn(kx[2], c0r, h);
            h = fma_rn(kx[3], c1r, h);
            h = fma_rn(kx[4], cp2, h);
        } else {  // even columns of a coarse row are coarse nodes: C = 0
            h = fma_rn(kx[1], cm1, mul_rn(kx[3], c1r));
        }
        // fine row 2 Y0 - 2 + r feeds coarse row Y0 + j with tap r - 2 j
#pragma unroll
        for (int j = 0; j < TY; ++j) {
            const int bb = r - 2 * j;
            if (bb >= 0 && bb <= 4) g[j] = fma_rn(FAST ? ku[bb] : __ldg(k1 + 5 * (Y0 + j) + bb), h, g[j]);
        }
    }
}

template <typename T, typename TW, bool HZ>
__global__ void __launch_bounds__(kStripThreads, 2) k_restrict_strip(RestrictParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr int TY = StripRows<T>::value;
    const T *__restrict__ A = static_cast<const T *>(p.A);
    TW *__restrict__ F = static_cast<TW *>(p.F);
    TW *__restrict__ V = static_cast<TW *>(p.V);
    const T *__restrict__ k0 = static_cast<const T *>(p.k0);
    const T *__restrict__ k1 = static_cast<const T *>(p.k1);
    const T *__restrict__ k2 = static_cast<const T *>(p.k2);
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int n1 = (int)p.n1, n2 = (int)p.n2;
    const int m0 = (int)p.m0, m1 = (int)p.m1, m2 = (int)p.m2;
    const int S = p.tiles_x, B = p.tiles_y;
    const int64_t plane_sz = (int64_t)n1 * n2, cplane = (int64_t)m1 * m2;

    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < p.nitems; item += gridDim.x * wpb) {
        const int s = item % S, rest = item / S;
        const int b = rest % B, c = rest / B;
        const int xown0 = kStripCols * s, yown = TY * b;
        const int X0 = min(xown0, m2 - kStripCols), Y0 = min(yown, m1 - TY);
        const int X = X0 - 1 + lane;  // lanes 0 and 31: neighbour columns only
        const bool active = lane >= 1 && lane <= kStripCols;
        const bool xown = active && X >= xown0;
        const int cx = 2 * X;
        T kx[5], ku[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) kx[t] = active ? k2[5 * X + t] : T(0);
        // fast path: the strip's coarse rows share one dim-1 stencil (the
        // level's interior rows are all equal and the strip holds no boundary
        // row), and its fine rows 2 Y0 - 2 .. 2 Y0 + 2 TY and columns
        // 2 X0 - 3 .. 2 X0 + 61 are inside the grid
        const bool uni = p.kuni1 && Y0 >= 1 && Y0 + TY <= m1 - 1 && 2 * (Y0 + TY) < n1 && X0 >= 2 &&
                         X0 + 31 < m2;
#pragma unroll
        for (int t = 0; t < 5; ++t) ku[t] = uni ? __ldg(k1 + 5 * Y0 + t) : T(0);

        const int Zs = HZ ? c * p.zchunk : 0;
        const int Ze = HZ ? (c == p.nzc - 1 ? m0 : Zs + p.zchunk) : 1;
        const int Zfirst = (HZ && Zs > 0) ? Zs - 1 : Zs;
        const int Zlast = HZ ? min(Ze, m0 - 1) : 0;

        T accP[TY], accC[TY], accN[TY];
#pragma unroll
        for (int j = 0; j < TY; ++j) accP[j] = accC[j] = accN[j] = T(0);
        (void)accN;

        auto store = [&](int Zo, const T (&acc)[TY]) {
            if (!xown) return;
            TW *f = F + (int64_t)Zo * cplane + X;
#pragma unroll
            for (int j = 0; j < TY; ++j)
                if (Y0 + j >= yown) f[(int64_t)(Y0 + j) * m2] = static_cast<TW>(acc[j]);
        };

        for (int Z = Zfirst; Z <= Zlast; ++Z) {
            T g[TY];
            const bool has_odd = HZ && Z >= 1 && Z >= Zs;
            const bool own_even = Z >= Zs && Z < Ze;
            if constexpr (HZ) {
                // odd plane 2Z-1: taps 3 of Z-1 and 1 of Z
                if (has_odd) {
                    const T *po = A + (int64_t)(2 * Z - 1) * plane_sz;
                    if (uni)
                        strip_plane<T, TW, TY, true, true>(po, n1, n2, Y0, cx, kx, ku, k1, g, false, V,
                                                           yown, m2, X, xown);
                    else
                        strip_plane<T, TW, TY, true, false>(po, n1, n2, Y0, cx, kx, ku, k1, g, false, V,
                                                            yown, m2, X, xown);
                    const T kzP3 = __ldg(k0 + 5 * (Z - 1) + 3), kzC1 = __ldg(k0 + 5 * Z + 1);
#pragma unroll
                    for (int j = 0; j < TY; ++j) {
                        accP[j] = fma_rn(kzP3, g[j], accP[j]);
                        accC[j] = fma_rn(kzC1, g[j], accC[j]);
                    }
                }
            }
            // even plane 2Z: taps 4 of Z-1, 2 of Z, 0 of Z+1
            const T *pe = A + (int64_t)(HZ ? 2 * Z : 0) * plane_sz;
            TW *vpe = V + (int64_t)(HZ ? Z : 0) * cplane;
            if (uni)
                strip_plane<T, TW, TY, false, true>(pe, n1, n2, Y0, cx, kx, ku, k1, g, own_even, vpe, yown,
                                                    m2, X, xown);
            else
                strip_plane<T, TW, TY, false, false>(pe, n1, n2, Y0, cx, kx, ku, k1, g, own_even, vpe,
                                                     yown, m2, X, xown);
            if constexpr (HZ) {
                const T kzP4 = (Z >= 1) ? __ldg(k0 + 5 * (Z - 1) + 4) : T(0);
                const T kzC2 = __ldg(k0 + 5 * Z + 2);
                const T kzN0 = (Z + 1 < m0) ? __ldg(k0 + 5 * (Z + 1)) : T(0);
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accP[j] = fma_rn(kzP4, g[j], accP[j]);
                    accC[j] = fma_rn(kzC2, g[j], accC[j]);
                    accN[j] = mul_rn(kzN0, g[j]);
                }
                // F(Z-1) is complete once the planes up to 2Z are in
                if (Z - 1 >= Zs && Z - 1 < Ze) store(Z - 1, accP);
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accP[j] = accC[j];
                    accC[j] = accN[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < TY; ++j) accC[j] = g[j];
            }
        }
        // the last coarse plane of the grid has no contributions beyond it
        const int Zend = HZ ? m0 - 1 : 0;
        if (Zlast == Zend && Zend >= Zs && Zend < Ze) {
            if constexpr (HZ) store(Zend, accP);
            else store(Zend, accC);
        }
    }
}

}  // namespace mg
