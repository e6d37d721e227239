// restrict.cuh -- fused coefficient + load-vector kernel (one level).
//
// For a level array A with node counts (n0, n1, n2) and coarse counts
// (m0, m1, m2) = ((n-1)/2 + 1), one pass computes
//   MODE_DEC: C = A - Pi_{l-1} A on N_l \ N_{l-1} (multilinear interpolation
//             from the even-index corners, Section II-A-1);
//   MODE_REC: C = A on N_l \ N_{l-1} (A already holds coefficients);
// and in both modes
//   F = (K_0 (x) K_1 (x) K_2) C,  K = P^T M_l (mass then transfer along each
//       dimension, a 5-point stencil per coarse node, Section III-A-2)
//   V = A restricted to N_{l-1} (compact).
// The kernel only reads A: tiles overlap in their halos, so writing
// coefficients in place here would race with neighbouring tiles that still
// need the original values.  The decomposition writes them afterwards
// (k_place), with the same explicitly rounded interpolation, so the stored
// coefficients are bit-identical to the C used here.
//
// Work item = (tile of TY x TX coarse nodes in dims 1,2) x (chunk of coarse
// planes in dim 0).  The CTA streams the fine planes of its chunk through
// shared memory (cp.async, one step ahead): each step handles the odd plane
// 2Z-1 and the even plane 2Z, so the z-direction of both the interpolation
// and the stencil reduces to rolling register accumulators.  A slab covers
// fine rows [2Y0-2, 2Y0+2TY] and columns [2X0-2, 2X0+2TX] (a 2-node halo on
// the low side and 1 node on the high side, the reach of the K stencil).
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kRestrictThreads = 256;

template <int ACT, int TY_, int TX>
struct RestrictGeom {
    static constexpr bool HZ = (ACT & 4) != 0;
    static constexpr bool HY = (ACT & 2) != 0;
    static constexpr int TY = HY ? TY_ : 1;
    static constexpr int RY = HY ? 2 * TY + 3 : 1;  // slab rows
    static constexpr int CX = 2 * TX + 3;           // slab columns
    static constexpr int PL = RY * CX;              // elements per slab
    static constexpr int ROFF = HY ? 2 : 0;         // slab row of fine row 2*Y0
    static constexpr int COFF = 2;                  // slab column of fine col 2*X0
    static constexpr int NT = kRestrictThreads;
    static constexpr int PPT = (TY * TX + NT - 1) / NT;  // owned coarse nodes per thread

    // shared memory layout, in elements of T
    static constexpr int OFF_SLAB = 0;                        // 4 slabs (2 steps x odd/even)
    static constexpr int OFF_I = 4 * PL;                      // 2 interpolant planes (DEC)
    static constexpr int OFF_H = OFF_I + 2 * PL;              // 2 x-restricted planes RY x TX
    static constexpr int OFF_TAB = OFF_H + 2 * RY * TX;       // weights and stencils
    static constexpr int TAB = 2 * CX + 2 * RY + 5 * TX + 5 * TY;
    static constexpr int TOTAL = OFF_TAB + TAB;
};

template <typename T, typename TW, int ACT, int MODE, int TY_, int TX>
__global__ void __launch_bounds__(kRestrictThreads)
k_restrict(RestrictParams p)
{
    using G = RestrictGeom<ACT, TY_, TX>;
    constexpr bool HZ = G::HZ, HY = G::HY;
    constexpr int TY = G::TY, RY = G::RY, CX = G::CX, PL = G::PL;
    constexpr int NT = G::NT, PPT = G::PPT;
    constexpr bool DEC = (MODE == MODE_DEC);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *slab = sm + G::OFF_SLAB;
    T *Ib = sm + G::OFF_I;
    T *Hx = sm + G::OFF_H;
    T *wxl = sm + G::OFF_TAB;
    T *wxr = wxl + CX;
    T *wyl = wxr + CX;
    T *wyr = wyl + RY;
    T *kx = wyr + RY;
    T *ky = kx + 5 * TX;

    T *A = static_cast<T *>(p.A);
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const T *w0 = static_cast<const T *>(p.w0);
    const T *w1 = static_cast<const T *>(p.w1);
    const T *w2 = static_cast<const T *>(p.w2);
    const T *k0 = static_cast<const T *>(p.k0);
    const T *k1 = static_cast<const T *>(p.k1);
    const T *k2 = static_cast<const T *>(p.k2);

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = NT / 32;
    const int64_t n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2;
    const int ntiles = p.tiles_y * p.tiles_x;

    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
        const int tile = item % ntiles;
        const int zc = item / ntiles;
        const int64_t Y0 = HY ? (int64_t)(tile / p.tiles_x) * TY : 0;
        const int64_t X0 = (int64_t)(tile % p.tiles_x) * TX;
        const int TYo = HY ? (int)min64(TY, m1 - Y0) : 1;
        const int TXo = (int)min64(TX, m2 - X0);
        const int64_t gy0 = HY ? 2 * Y0 - 2 : 0;
        const int64_t gx0 = 2 * X0 - 2;
        const int64_t Zs = HZ ? (int64_t)zc * p.zchunk : 0;
        const int64_t Ze = HZ ? min64(m0, Zs + p.zchunk) : 1;
        const int64_t Zfirst = (HZ && Zs > 0) ? Zs - 1 : Zs;
        const int64_t Zlast = HZ ? min64(Ze, m0 - 1) : 0;

        __syncthreads();  // the previous item is done with shared memory

        // per-tile weights and stencil rows
        for (int c = tid; c < CX; c += NT) {
            const int64_t gx = gx0 + c;
            const bool odd = (gx > 0) && (gx < n2 - 1) && (gx & 1);
            wxl[c] = odd ? w2[2 * gx] : T(0);
            wxr[c] = odd ? w2[2 * gx + 1] : T(0);
        }
        if constexpr (HY) {
            for (int r = tid; r < RY; r += NT) {
                const int64_t gy = gy0 + r;
                const bool odd = (gy > 0) && (gy < n1 - 1) && (gy & 1);
                wyl[r] = odd ? w1[2 * gy] : T(0);
                wyr[r] = odd ? w1[2 * gy + 1] : T(0);
            }
            for (int e = tid; e < 5 * TY; e += NT) {
                const int Y = e / 5;
                ky[e] = (Y < TYo) ? k1[5 * (Y0 + Y) + (e % 5)] : T(0);
            }
        }
        for (int e = tid; e < 5 * TX; e += NT) {
            const int X = e / 5;
            kx[e] = (X < TXo) ? k2[5 * (X0 + X) + (e % 5)] : T(0);
        }

        // Issue the loads of the fine planes of step Z into slab pair s.
        auto issue = [&](int64_t Z, int s) {
            const bool odd_plane = HZ && Z >= 1 && Z >= Zs;
            for (int q = 0; q < 2; ++q) {
                if (q == 0 && !odd_plane) continue;
                const int64_t z = HZ ? (q == 0 ? 2 * Z - 1 : 2 * Z) : 0;
                T *dst = slab + (2 * s + q) * PL;
                const T *plane = A + z * n1 * n2;
                for (int e = tid; e < PL; e += NT) {
                    const int r = e / CX, c = e - (e / CX) * CX;
                    const int64_t gy = gy0 + r, gx = gx0 + c;
                    const bool ok = (gy >= 0) && (gy < n1) && (gx >= 0) && (gx < n2);
                    const T *src = ok ? plane + gy * n2 + gx : A;
                    cp_async_elem(dst + e, src, ok);
                }
            }
            cp_async_commit();
        };

        issue(Zfirst, 0);
        if (Zfirst + 1 <= Zlast) issue(Zfirst + 1, 1);
        else cp_async_commit();

        T accP[PPT], accC[PPT], accN[PPT];
#pragma unroll
        for (int i = 0; i < PPT; ++i) accP[i] = accC[i] = accN[i] = T(0);

        for (int64_t Z = Zfirst; Z <= Zlast; ++Z) {
            const int s = (int)((Z - Zfirst) & 1);
            const bool has_odd = HZ && Z >= 1 && Z >= Zs;
            const bool own_even = (Z >= Zs) && (Z < Ze);
            T *So = slab + (2 * s) * PL;
            T *Se = slab + (2 * s + 1) * PL;
            T *Icur = Ib + s * PL;
            T *Iprev = Ib + (1 - s) * PL;

            cp_async_wait<1>();
            __syncthreads();

            if constexpr (DEC) {
                // interpolant of the even plane from its even-even nodes
                for (int e = tid; e < PL; e += NT) {
                    const int r = e / CX, c = e - (e / CX) * CX;
                    const bool ro = HY && (r & 1), co = (c & 1);
                    T iv;
                    if (!ro && !co) {
                        iv = Se[e];
                    } else if (!ro) {
                        iv = lerp2(wxl[c], Se[e - 1], wxr[c], Se[e + 1]);
                    } else if (!co) {
                        iv = lerp2(wyl[r], Se[e - CX], wyr[r], Se[e + CX]);
                    } else {
                        iv = lerp2(wyl[r], lerp2(wxl[c], Se[e - CX - 1], wxr[c], Se[e - CX + 1]), wyr[r],
                                   lerp2(wxl[c], Se[e + CX - 1], wxr[c], Se[e + CX + 1]));
                    }
                    Icur[e] = iv;
                }
                __syncthreads();
                // coefficients in place; the even-even nodes of the even plane keep u
                T wzl = T(0), wzr = T(0);
                if (has_odd) {
                    wzl = w0[2 * (2 * Z - 1)];
                    wzr = w0[2 * (2 * Z - 1) + 1];
                }
                for (int e = tid; e < PL; e += NT) {
                    const int r = e / CX, c = e - (e / CX) * CX;
                    const bool ee = !(HY && (r & 1)) && !(c & 1);
                    if (!ee) Se[e] = sub_rn(Se[e], Icur[e]);
                    if (has_odd) So[e] = sub_rn(So[e], lerp2(wzl, Iprev[e], wzr, Icur[e]));
                }
                __syncthreads();
            }

            // coarse values of the owned coarse nodes
            if (own_even) {
                TW *vrow = V + (HZ ? Z * m1 * m2 : 0);
                for (int Y = warp; Y < TYo; Y += NWARP) {
                    const int r = G::ROFF + 2 * Y;
                    for (int X = lane; X < TXo; X += 32)
                        vrow[(Y0 + Y) * m2 + X0 + X] = static_cast<TW>(Se[r * CX + G::COFF + 2 * X]);
                }
            }

            // x-direction stencil of both planes: Hx[r][X] = sum_t kx[X][t] C[r][2X+t]
            T *Ho = Hx;
            T *He = Hx + RY * TX;
            for (int e = tid; e < RY * TX; e += NT) {
                const int r = e / TX, X = e - (e / TX) * TX;
                const T *ce = Se + r * CX + 2 * X;
                const T *kk = kx + 5 * X;
                T he;
                if (!(HY && (r & 1))) {
                    he = kk[1] * ce[1] + kk[3] * ce[3];  // even row of the even plane: C = 0 at even columns
                } else {
                    he = kk[0] * ce[0] + kk[1] * ce[1] + kk[2] * ce[2] + kk[3] * ce[3] + kk[4] * ce[4];
                }
                He[e] = he;
                if (has_odd) {
                    const T *co = So + r * CX + 2 * X;
                    Ho[e] = kk[0] * co[0] + kk[1] * co[1] + kk[2] * co[2] + kk[3] * co[3] + kk[4] * co[4];
                }
            }
            __syncthreads();

            // y-direction stencil and z accumulation of the owned coarse nodes
            T kzP[5], kzC[5], kzN[5];
            if constexpr (HZ) {
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    kzP[t] = (Z >= 1) ? k0[5 * (Z - 1) + t] : T(0);
                    kzC[t] = k0[5 * Z + t];
                    kzN[t] = (Z + 1 < m0) ? k0[5 * (Z + 1) + t] : T(0);
                }
            }
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int pos = tid + i * NT;
                if (pos >= TY * TX) break;
                const int Y = pos / TX, X = pos - (pos / TX) * TX;
                T ge, go = T(0);
                if constexpr (HY) {
                    const T *kk = ky + 5 * Y;
                    const T *he = He + (2 * Y) * TX + X;
                    ge = kk[0] * he[0] + kk[1] * he[TX] + kk[2] * he[2 * TX] + kk[3] * he[3 * TX] +
                         kk[4] * he[4 * TX];
                    if (has_odd) {
                        const T *ho = Ho + (2 * Y) * TX + X;
                        go = kk[0] * ho[0] + kk[1] * ho[TX] + kk[2] * ho[2 * TX] + kk[3] * ho[3 * TX] +
                             kk[4] * ho[4 * TX];
                    }
                } else {
                    ge = He[X];
                }
                if constexpr (HZ) {
                    accP[i] += kzP[3] * go + kzP[4] * ge;
                    accC[i] += kzC[1] * go + kzC[2] * ge;
                    accN[i] += kzN[0] * ge;
                } else {
                    accC[i] = ge;
                }
            }

            if constexpr (HZ) {
                // F(Z-1) is complete once the planes up to 2Z are in
                if (Z - 1 >= Zs && Z - 1 < Ze) {
#pragma unroll
                    for (int i = 0; i < PPT; ++i) {
                        const int pos = tid + i * NT;
                        if (pos >= TY * TX) break;
                        const int Y = pos / TX, X = pos - (pos / TX) * TX;
                        if (Y < TYo && X < TXo)
                            F[((Z - 1) * m1 + Y0 + Y) * m2 + X0 + X] = static_cast<TW>(accP[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < PPT; ++i) {
                    accP[i] = accC[i];
                    accC[i] = accN[i];
                    accN[i] = T(0);
                }
            }

            __syncthreads();  // slabs of this step may now be refilled
            if (Z + 2 <= Zlast) issue(Z + 2, s);
            else cp_async_commit();
        }

        // the last coarse plane of the grid has no contributions beyond it
        const int64_t Zend = HZ ? m0 - 1 : 0;
        if (Zlast == Zend && Zend >= Zs && Zend < Ze) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int pos = tid + i * NT;
                if (pos >= TY * TX) break;
                const int Y = pos / TX, X = pos - (pos / TX) * TX;
                if (Y < TYo && X < TXo)
                    F[(Zend * m1 + Y0 + Y) * m2 + X0 + X] = static_cast<TW>(HZ ? accP[i] : accC[i]);
            }
        }
        cp_async_wait<0>();
    }
}

}  // namespace mg
