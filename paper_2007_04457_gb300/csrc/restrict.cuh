// restrict.cuh -- load vector and coarse gather of one level (both directions).
//
// The level array A holds the coefficients C on N_l \ N_{l-1} (the
// decomposition writes them before this pass) and coarse values on N_{l-1}.
// One pass computes
//   F = (K_0 (x) K_1 (x) K_2) C,  C = A on N_l \ N_{l-1}, 0 on N_{l-1}
//       (K = P^T M_l: mass then transfer along each dimension, a 5-point
//       stencil per coarse node, Section III-A-2)
//   V = A restricted to N_{l-1} (compact)
// and only reads A.
//
// Two- and three-dimensional levels (k_restrict): work item = tile of TY x
// 64 coarse nodes in dims (1, 2) (the last tile of a
// dimension absorbs the final node, so it may hold TY+1 x 65) x a chunk of
// coarse planes in dim 0.  The CTA streams the fine planes of its chunk
// through shared memory with cp.async, one step ahead; each step handles the
// odd plane 2Z-1 and the even plane 2Z, so the dim-0 part of the stencil
// reduces to rolling register accumulators.
//
// Every warp shuffle below runs in all 32 lanes (full mask) and the lanes
// that need a halo value select it afterwards; a shuffle under a lane
// condition would leave the warp waiting for the lanes that skipped it.
//
// Thread mapping inside a plane: warp w takes slab rows w, w+8, ...; lane L
// takes the four fine columns 4L..4L+3 of the tile (coarse columns 2L and
// 2L+1), so the row loads are 128-bit shared-memory loads, and the 5-point
// dim-2 stencil takes its two left and one right neighbour values from the
// adjacent lanes by shuffles.  Lane 0 also covers the two fine columns left
// of the tile and lane 31 the one on its right (and the 65th coarse column
// of a last tile).  The dim-1 stencil then reads the dim-2-restricted rows
// from shared memory.
// One-dimensional levels (k_restrict1d): one thread per coarse node.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kRestrictThreads = 256;
constexpr int kRestrictTX = 64;  // coarse columns per tile (+1 in a last tile)

template <typename T, int ACT, int TY_>
struct RestrictGeom {
    static constexpr bool HZ = (ACT & 4) != 0;
    static constexpr bool HY = (ACT & 2) != 0;
    static constexpr int TY = HY ? TY_ : 1;
    static constexpr int RYM = HY ? 2 * TY + 5 : 1;   // slab rows, sized for a TY+1 last tile
    static constexpr int SP = 136;                    // slab pitch: fine cols 2X0-4 .. 2X0+131
    static constexpr int HP = 68;                     // pitch of the dim-2-restricted rows
    static constexpr int NT = kRestrictThreads;
    static constexpr int NWARP = NT / 32;
    static constexpr int OUTS = (HY ? TY + 1 : 1) * HP;    // output slots per plane pair
    static constexpr int PPT = (OUTS + NT - 1) / NT;       // output slots per thread

    // shared memory layout, in elements of T
    static constexpr int OFF_SLAB = 0;                   // 4 slabs
    static constexpr int OFF_H = OFF_SLAB + 4 * RYM * SP;  // 2 restricted planes
    static constexpr int OFF_KY = OFF_H + 2 * RYM * HP;    // dim-1 stencil rows
    static constexpr int TOTAL = OFF_KY + 5 * (TY + 1);
};

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        const double2 b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
}

template <typename T>
__device__ __forceinline__ T shfl_dn(T v)
{
    return __shfl_down_sync(0xffffffffu, v, 1);
}

template <typename T>
__device__ __forceinline__ T shfl_upw(T v)
{
    return __shfl_up_sync(0xffffffffu, v, 1);
}

// 5-point dim-2 stencil of the two coarse columns of a lane from the lane's
// four C values, its left neighbour's last two (cl2, cl3) and its right
// neighbour's first (crr).
template <typename T>
__device__ __forceinline__ void stencil2(const T (&ka)[5], const T (&kb)[5], T cl2, T cl3, const T (&c)[4],
                                         T crr, T &ha, T &hb)
{
    ha = fma_rn(ka[0], cl2, mul_rn(ka[1], cl3));
    ha = fma_rn(ka[2], c[0], ha);
    ha = fma_rn(ka[3], c[1], ha);
    ha = fma_rn(ka[4], c[2], ha);
    hb = fma_rn(kb[0], c[0], mul_rn(kb[1], c[1]));
    hb = fma_rn(kb[2], c[2], hb);
    hb = fma_rn(kb[3], c[3], hb);
    hb = fma_rn(kb[4], crr, hb);
}

// Resident blocks per SM the register allocation is sized for: 4 for the
// small FP32 tiles (49 KB of shared memory), 2 otherwise.
template <typename T, int TY_>
constexpr int restrict_min_blocks()
{
    return (sizeof(T) == 4 && TY_ <= 4) ? 4 : 2;
}

template <typename T, typename TW, int ACT, int TY_>
__global__ void __launch_bounds__(kRestrictThreads, (restrict_min_blocks<T, TY_>()))
k_restrict(RestrictParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    using G = RestrictGeom<T, ACT, TY_>;
    constexpr bool HZ = G::HZ, HY = G::HY;
    constexpr int TY = G::TY, RYM = G::RYM, SP = G::SP, HP = G::HP;
    constexpr int NT = G::NT, NWARP = G::NWARP, PPT = G::PPT;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *slab = sm + G::OFF_SLAB;
    T *Hb = sm + G::OFF_H;
    T *sky = sm + G::OFF_KY;

    const T *A = static_cast<const T *>(p.A);
    TW *F = static_cast<TW *>(p.F);
    TW *V = static_cast<TW *>(p.V);
    const T *k0 = static_cast<const T *>(p.k0);
    const T *k1 = static_cast<const T *>(p.k1);
    const T *k2 = static_cast<const T *>(p.k2);

    const int tid = threadIdx.x;
    const int L = tid & 31, warp = tid >> 5;
    const int64_t n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2;
    const int ntiles = p.tiles_y * p.tiles_x;
    const uint64_t pol = policy_evict_first();  // the level array is streamed once

    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
        const int tile = item % ntiles;
        const int zc = item / ntiles;
        const int ty = HY ? tile / p.tiles_x : 0;
        const int tx = tile % p.tiles_x;
        const int64_t Y0 = (int64_t)ty * TY;
        const int64_t X0 = (int64_t)tx * kRestrictTX;
        const int TYo = HY ? (ty == p.tiles_y - 1 ? (int)(m1 - Y0) : TY) : 1;
        const int TXo = (tx == p.tiles_x - 1) ? (int)(m2 - X0) : kRestrictTX;
        const bool wide = TXo > kRestrictTX;  // a last tile with the 65th coarse column
        const int NO = TYo * TXo;             // coarse nodes of the tile per plane
        const int RY = HY ? 2 * TYo + 3 : 1;
        const int64_t gy0 = HY ? 2 * Y0 - 2 : 0;   // fine row of slab row 0
        const int64_t gx0 = 2 * X0 - 4;            // fine column of slab column 0
        const int64_t Zs = HZ ? (int64_t)zc * p.zchunk : 0;
        const int64_t Ze = HZ ? (zc == p.nzc - 1 ? m0 : Zs + p.zchunk) : 1;
        const int64_t Zfirst = (HZ && Zs > 0) ? Zs - 1 : Zs;
        const int64_t Zlast = HZ ? min64(Ze, m0 - 1) : 0;

        // per-lane stencil rows of coarse columns 2L, 2L+1 (and lane 31's
        // column 64 of a 65-wide tile)
        T ka[5], kb[5], kc[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            ka[t] = (2 * L < TXo) ? k2[5 * (X0 + 2 * L) + t] : T(0);
            kb[t] = (2 * L + 1 < TXo) ? k2[5 * (X0 + 2 * L + 1) + t] : T(0);
            kc[t] = (L == 31 && TXo > 64) ? k2[5 * (X0 + 64) + t] : T(0);
        }
        // column validity of the lane's load slots L + 32k
        unsigned colmask = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int s = L + 32 * k;
            const int64_t gx = gx0 + s;
            if (s < SP && gx >= 0 && gx < n2) colmask |= 1u << k;
        }

        __syncthreads();  // the previous item is done with shared memory
        if constexpr (HY) {
            for (int e = tid; e < 5 * (TY + 1); e += NT) {
                const int Y = e / 5;
                sky[e] = (Y < TYo) ? k1[5 * (Y0 + Y) + (e % 5)] : T(0);
            }
        }

        // Loads of the fine planes of step Z into slab pair s.
        auto issue = [&](int64_t Z, int s) {
            const bool odd_plane = HZ && Z >= 1 && Z >= Zs;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q == 0 && !odd_plane) continue;
                const int64_t z = HZ ? (q == 0 ? 2 * Z - 1 : 2 * Z) : 0;
                T *dst = slab + (2 * s + q) * (RYM * SP);
                const T *plane = A + z * n1 * n2;
                for (int r = warp; r < RY; r += NWARP) {
                    const int64_t gy = gy0 + r;
                    const bool rok = (gy >= 0) && (gy < n1);
                    const T *src = plane + (rok ? gy : 0) * n2 + gx0;
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const int s2 = L + 32 * k;
                        if (s2 < SP) {
                            const bool ok = rok && ((colmask >> k) & 1u);
                            cp_async_elem_hint(dst + r * SP + s2, ok ? src + s2 : A, ok, pol);
                        }
                    }
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
        // output slot i of this thread: coarse node pos = tid + i NT of the
        // tile's TYo x TXo nodes, row-major (the same every step of the tile);
        // slots run in order, so the first one past the tile ends the loop,
        // and an interior 16 x 64 tile fills exactly four slots per thread
        auto out_slot = [&](int i, int &Y, int &X) -> bool {
            const int pos = tid + i * NT;
            if (pos >= NO) return false;
            Y = (TXo == kRestrictTX) ? (pos >> 6) : pos / TXo;
            X = pos - Y * TXo;
            return true;
        };

        for (int64_t Z = Zfirst; Z <= Zlast; ++Z) {
            const int s = (int)((Z - Zfirst) & 1);
            const bool has_odd = HZ && Z >= 1 && Z >= Zs;
            const bool own_even = (Z >= Zs) && (Z < Ze);
            const T *So = slab + (2 * s) * (RYM * SP);
            const T *Se = slab + (2 * s + 1) * (RYM * SP);
            T *He = Hb + RYM * HP;
            T *Ho = Hb;

            cp_async_wait<1>();
            __syncthreads();

            // ---- passes over the rows of the two planes (warp-private rows)
            for (int r = warp; r < RY; r += NWARP) {
                const bool ro = HY && (r & 1);
                const int rb = r * SP + 4 * L + 4;  // slab index of the lane's first column
                T u[4], C[4], chl2, chl1, ch128;    // halo C: cols -2, -1 (lane 0), 128 (lane 31)
                ld4(Se + rb, u);
                const T uh128 = Se[r * SP + 132];
                const T uhm2 = Se[r * SP + 2], uhm1 = Se[r * SP + 3];
                // even plane: coarse nodes (even row, even column) carry no coefficient
                {
                    C[0] = ro ? u[0] : T(0);
                    C[1] = u[1];
                    C[2] = ro ? u[2] : T(0);
                    C[3] = u[3];
                    chl2 = ro ? uhm2 : T(0);
                    chl1 = uhm1;
                    ch128 = ro ? uh128 : T(0);
                }
                // coarse values of the owned coarse nodes (even row of an owned even plane)
                if (own_even && !ro) {
                    const int Yl = HY ? (r - 2) / 2 : 0;
                    if (r >= (HY ? 2 : 0) && Yl < TYo) {
                        TW *vrow = V + ((HZ ? Z : 0) * m1 + Y0 + Yl) * m2 + X0;
                        if (2 * L < TXo) vrow[2 * L] = static_cast<TW>(u[0]);
                        if (2 * L + 1 < TXo) vrow[2 * L + 1] = static_cast<TW>(u[2]);
                        if (L == 31 && TXo > 64) vrow[64] = static_cast<TW>(uh128);
                    }
                }
                // dim-2 stencil of the even plane
                {
                    T cl2 = shfl_upw(C[2]), cl3 = shfl_upw(C[3]);
                    const T cr0 = shfl_dn(C[0]);
                    if (L == 0) { cl2 = chl2; cl3 = chl1; }
                    const T crr = (L == 31) ? ch128 : cr0;
                    T ha, hb;
                    if (ro) {
                        stencil2(ka, kb, cl2, cl3, C, crr, ha, hb);
                    } else {  // C[0], C[2], cl2, crr are 0: the nonzero taps only
                        ha = fma_rn(ka[3], C[1], mul_rn(ka[1], cl3));
                        hb = fma_rn(kb[3], C[3], mul_rn(kb[1], C[1]));
                    }
                    T *hrow = He + r * HP;
                    hrow[2 * L] = ha;
                    hrow[2 * L + 1] = hb;
                    if (wide && L == 31)
                        hrow[64] = fma_rn(kc[2], ch128, fma_rn(kc[0], C[2], mul_rn(kc[1], C[3])));
                }
                // odd plane: every node is a coefficient node
                if (has_odd) {
                    T v[4];
                    ld4(So + rb, v);
                    const T ohm2 = So[r * SP + 2], ohm1 = So[r * SP + 3], oh128 = So[r * SP + 132];
                    T cl2 = shfl_upw(v[2]), cl3 = shfl_upw(v[3]);
                    const T cr0 = shfl_dn(v[0]);
                    if (L == 0) { cl2 = ohm2; cl3 = ohm1; }
                    const T crr = (L == 31) ? oh128 : cr0;
                    T ha, hb;
                    stencil2(ka, kb, cl2, cl3, v, crr, ha, hb);
                    T *hrow = Ho + r * HP;
                    hrow[2 * L] = ha;
                    hrow[2 * L + 1] = hb;
                    if (wide && L == 31)
                        hrow[64] = fma_rn(kc[2], oh128, fma_rn(kc[0], v[2], mul_rn(kc[1], v[3])));
                }
            }
            __syncthreads();  // restricted rows complete; the slabs of this step are free
            if (Z + 2 <= Zlast) issue(Z + 2, s);
            else cp_async_commit();

            // ---- dim-1 stencil and dim-0 accumulation of the owned coarse nodes
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
                int Y, X;
                if (!out_slot(i, Y, X)) break;
                T ge, go = T(0);
                if constexpr (HY) {
                    const T *kk = sky + 5 * Y;
                    const T *he = He + (2 * Y) * HP + X;
                    ge = fma_rn(kk[0], he[0], mul_rn(kk[1], he[HP]));
                    ge = fma_rn(kk[2], he[2 * HP], ge);
                    ge = fma_rn(kk[3], he[3 * HP], ge);
                    ge = fma_rn(kk[4], he[4 * HP], ge);
                    if (has_odd) {
                        const T *ho = Ho + (2 * Y) * HP + X;
                        go = fma_rn(kk[0], ho[0], mul_rn(kk[1], ho[HP]));
                        go = fma_rn(kk[2], ho[2 * HP], go);
                        go = fma_rn(kk[3], ho[3 * HP], go);
                        go = fma_rn(kk[4], ho[4 * HP], go);
                    }
                } else {
                    ge = He[X];
                }
                if constexpr (HZ) {
                    accP[i] = fma_rn(kzP[3], go, fma_rn(kzP[4], ge, accP[i]));
                    accC[i] = fma_rn(kzC[1], go, fma_rn(kzC[2], ge, accC[i]));
                    accN[i] = fma_rn(kzN[0], ge, accN[i]);
                } else {
                    accC[i] = ge;
                }
            }
            if constexpr (HZ) {
                // F(Z-1) is complete once the planes up to 2Z are in
                if (Z - 1 >= Zs && Z - 1 < Ze) {
#pragma unroll
                    for (int i = 0; i < PPT; ++i) {
                        int Y, X;
                        if (!out_slot(i, Y, X)) break;
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
        }

        // the last coarse plane of the grid has no contributions beyond it
        const int64_t Zend = HZ ? m0 - 1 : 0;
        if (Zlast == Zend && Zend >= Zs && Zend < Ze) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                int Y, X;
                if (!out_slot(i, Y, X)) break;
                F[(Zend * m1 + Y0 + Y) * m2 + X0 + X] = static_cast<TW>(HZ ? accP[i] : accC[i]);
            }
        }
        cp_async_wait<0>();
    }
}

// One thread per coarse node I (both directions: the decomposition writes
// its coefficients before this pass).
template <typename T, typename TW>
__global__ void __launch_bounds__(256) k_restrict1d(RestrictParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    const T *__restrict__ A = static_cast<const T *>(p.A);
    TW *__restrict__ F = static_cast<TW *>(p.F);
    TW *__restrict__ V = static_cast<TW *>(p.V);
    const T *__restrict__ k2 = static_cast<const T *>(p.k2);
    const int64_t n2 = p.n2, m2 = p.m2;
    auto coef = [&](int64_t j) -> T {  // C at the odd fine node j (0 outside the grid)
        return (j < 1 || j > n2 - 2) ? T(0) : A[j];
    };
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < m2;
         I += (int64_t)gridDim.x * blockDim.x) {
        const T cl = coef(2 * I - 1), cr = coef(2 * I + 1);
        F[I] = static_cast<TW>(fma_rn(k2[5 * I + 3], cr, mul_rn(k2[5 * I + 1], cl)));
        V[I] = static_cast<TW>(A[2 * I]);
    }
}

}  // namespace mg
