// adjoint.cuh -- kernels of the transposed level maps (decomposition and
// recomposition are linear; their transposes back-propagate gradients).
//
// With o = nodes of N_l \ N_{l-1}, e = nodes of N_{l-1}, K = P^T M_l (the
// 5-point restriction stencil of the forward maps; M_l P = K^T because M_l
// is symmetric) and Pi^T the transposed interpolation:
//   decomposition step  o' = o - Pi e,  e' = e + M_{l-1}^{-1} K (o - Pi e)
//   its transpose       w = o_bar' + [K^T M_{l-1}^{-1} e_bar']_o,
//                       o_bar = w,  e_bar = e_bar' - Pi^T w
//   recomposition step  e_new = e - M_{l-1}^{-1} K o,  o_new = o + Pi e_new
//   its transpose       e_tot = e_bar_new + Pi^T o_bar_new,
//                       o_bar = o_bar_new - [K^T M_{l-1}^{-1} e_tot]_o,
//                       e_bar = e_tot
// (Section II-A, Eq. 1-2, transposed; M_{l-1} is symmetric).
//
// k_gather:  compact V <- the N_{l-1} nodes of the level array.
// k_adj_odd: A(o) <- A(o) + s (K^T z)(o) for every node of N_l \ N_{l-1}.
// k_adj_even: A(e) <- B(e) + s (Pi^T A|_o)(e) for every node of N_{l-1}, B
//   either A itself or the compact V; reads only nodes of N_l \ N_{l-1} and
//   writes only nodes of N_{l-1}, so threads never race.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kAdjThreads = 256;

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kAdjThreads) k_gather(PlaceParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    const T *__restrict__ A = static_cast<const T *>(p.A);
    TW *__restrict__ V = const_cast<TW *>(static_cast<const TW *>(p.V));
    const int64_t X = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= p.m2) return;
    for (int64_t Z = blockIdx.z; Z < p.m0; Z += gridDim.z) {
        const int64_t z = HZ ? 2 * Z : 0;
        for (int64_t Y = blockIdx.y; Y < p.m1; Y += gridDim.y) {
            const int64_t y = HY ? 2 * Y : 0;
            V[(Z * p.m1 + Y) * p.m2 + X] = static_cast<TW>(A[(z * p.n1 + y) * p.n2 + 2 * X]);
        }
    }
}

// Coarse neighbours of fine index j along one dimension with their K^T
// weights: even j = 2I: I-1 (t=4), I (t=2), I+1 (t=0); odd j = 2I+1:
// I (t=3), I+1 (t=1).  Returns the count (<= 3).
template <typename TW>
__device__ __forceinline__ int kt_support(int64_t j, int64_t m, const TW *k, int64_t (&I)[3], TW (&w)[3])
{
    int c = 0;
    if (!(j & 1)) {
        const int64_t I0 = j >> 1;
        if (I0 - 1 >= 0) { I[c] = I0 - 1; w[c] = k[5 * (I0 - 1) + 4]; ++c; }
        I[c] = I0; w[c] = k[5 * I0 + 2]; ++c;
        if (I0 + 1 < m) { I[c] = I0 + 1; w[c] = k[5 * (I0 + 1)]; ++c; }
    } else {
        const int64_t I0 = j >> 1;
        I[c] = I0; w[c] = k[5 * I0 + 3]; ++c;
        if (I0 + 1 < m) { I[c] = I0 + 1; w[c] = k[5 * (I0 + 1) + 1]; ++c; }
    }
    return c;
}

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kAdjThreads) k_adj_odd(AdjParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ Z = static_cast<const TW *>(p.Z);
    const TW *k0 = static_cast<const TW *>(p.k0);
    const TW *k1 = static_cast<const TW *>(p.k1);
    const TW *k2 = static_cast<const TW *>(p.k2);
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.n2) return;
    int64_t Ix[3];
    TW wx[3];
    const int cx = kt_support(x, p.m2, k2, Ix, wx);
    for (int64_t z = blockIdx.z; z < p.n0; z += gridDim.z) {
        int64_t Iz[3] = {0, 0, 0};
        TW wz[3] = {TW(1), TW(0), TW(0)};
        const int cz = HZ ? kt_support(z, p.m0, k0, Iz, wz) : 1;
        for (int64_t y = blockIdx.y; y < p.n1; y += gridDim.y) {
            const bool odd = (x & 1) || (HY && (y & 1)) || (HZ && (z & 1));
            if (!odd) continue;
            int64_t Iy[3] = {0, 0, 0};
            TW wy[3] = {TW(1), TW(0), TW(0)};
            const int cy = HY ? kt_support(y, p.m1, k1, Iy, wy) : 1;
            TW g = TW(0);
            for (int a = 0; a < cz; ++a) {
                TW gy = TW(0);
                for (int b = 0; b < cy; ++b) {
                    const TW *zr = Z + (Iz[a] * p.m1 + Iy[b]) * p.m2;
                    TW gx = TW(0);
                    for (int c = 0; c < cx; ++c) gx += wx[c] * zr[Ix[c]];
                    gy += wy[b] * gx;
                }
                g += wz[a] * gy;
            }
            T *pa = A + (z * p.n1 + y) * p.n2 + x;
            const TW a = static_cast<TW>(*pa);
            *pa = static_cast<T>(p.sign > 0 ? a + g : a - g);
        }
    }
}

// Interpolation weights of the fine neighbours of coarse index E along one
// dimension: j = 2E-1 (E is its right corner: weight wr), j = 2E (weight 1,
// an even node in this dimension), j = 2E+1 (E is its left corner: wl).
template <typename TW, typename T>
__device__ __forceinline__ int pt_support(int64_t E, int64_t n, const T *w, int64_t (&j)[3], TW (&wt)[3])
{
    int c = 0;
    const int64_t f = 2 * E;
    if (f - 1 >= 1) { j[c] = f - 1; wt[c] = static_cast<TW>(w[2 * (f - 1) + 1]); ++c; }
    j[c] = f; wt[c] = TW(1); ++c;
    if (f + 1 <= n - 2) { j[c] = f + 1; wt[c] = static_cast<TW>(w[2 * (f + 1)]); ++c; }
    return c;
}

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(kAdjThreads) k_adj_even(AdjParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ B = static_cast<const TW *>(p.Z);  // compact base, or null: A itself
    const T *w0 = static_cast<const T *>(p.w0);
    const T *w1 = static_cast<const T *>(p.w1);
    const T *w2 = static_cast<const T *>(p.w2);
    const int64_t X = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= p.m2) return;
    int64_t jx[3];
    TW wx[3];
    const int cx = pt_support<TW>(X, p.n2, w2, jx, wx);
    for (int64_t Zc = blockIdx.z; Zc < p.m0; Zc += gridDim.z) {
        int64_t jz[3] = {0, 0, 0};
        TW wz[3] = {TW(1), TW(0), TW(0)};
        const int cz = HZ ? pt_support<TW>(Zc, p.n0, w0, jz, wz) : 1;
        for (int64_t Yc = blockIdx.y; Yc < p.m1; Yc += gridDim.y) {
            int64_t jy[3] = {0, 0, 0};
            TW wy[3] = {TW(1), TW(0), TW(0)};
            const int cy = HY ? pt_support<TW>(Yc, p.n1, w1, jy, wy) : 1;
            const int64_t ze = HZ ? 2 * Zc : 0, ye = HY ? 2 * Yc : 0;
            TW s = TW(0);
            for (int a = 0; a < cz; ++a) {
                for (int b = 0; b < cy; ++b) {
                    const T *row = A + (jz[a] * p.n1 + jy[b]) * p.n2;
                    const TW wab = wz[a] * wy[b];
                    for (int c = 0; c < cx; ++c) {
                        if (jz[a] == ze && jy[b] == ye && jx[c] == 2 * X) continue;  // the node itself
                        s += wab * wx[c] * static_cast<TW>(row[jx[c]]);
                    }
                }
            }
            T *pe = A + (ze * p.n1 + ye) * p.n2 + 2 * X;
            const TW base = B ? B[(Zc * p.m1 + Yc) * p.m2 + X] : static_cast<TW>(*pe);
            *pe = static_cast<T>(p.sign > 0 ? base + s : base - s);
        }
    }
}

// k_adj_odd2 (2D/3D): the same map as k_adj_odd, separably.  A warp item is a
// pair of fine planes (2Zp, 2Zp + 1) x a pair of fine rows (2Yp, 2Yp + 1);
// the K^T stencils of dims 0 and 1 reach the same 3 x 3 coarse rows
// (Iz, Iy in {Zp-1, Zp, Zp+1} x {Yp-1, Yp, Yp+1}) from all four fine rows,
// so the warp folds them per coarse column into four rows R in shared memory
// (one per fine row, with that row's dim-0 and dim-1 weights) and then
// applies the dim-2 stencil per fine column: about one coarse load per fine
// node instead of up to 27.
constexpr int kAdj2Warps = 4;

template <typename TW>
__device__ __forceinline__ void kt_pair(int64_t P, int64_t m, const TW *k, TW (&w)[2][3])
{
    // fine 2P (even): coarse P-1 (tap 4), P (tap 2), P+1 (tap 0);
    // fine 2P+1 (odd): coarse P (tap 3), P+1 (tap 1); slot a <-> coarse P-1+a
    w[0][0] = (P - 1 >= 0) ? k[5 * (P - 1) + 4] : TW(0);
    w[0][1] = k[5 * P + 2];
    w[0][2] = (P + 1 < m) ? k[5 * (P + 1)] : TW(0);
    w[1][0] = TW(0);
    w[1][1] = k[5 * P + 3];
    w[1][2] = (P + 1 < m) ? k[5 * (P + 1) + 1] : TW(0);
}

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(32 * kAdj2Warps) k_adj_odd2(AdjParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ Zc = static_cast<const TW *>(p.Z);
    const TW *k0 = static_cast<const TW *>(p.k0);
    const TW *k1 = static_cast<const TW *>(p.k1);
    const TW *k2 = static_cast<const TW *>(p.k2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TW *R = reinterpret_cast<TW *>(smem_raw) + (size_t)warp * 4 * m2;  // R[pz][py][X]
    const int64_t zp_n = HZ ? (n0 + 1) / 2 : 1, yp_n = (n1 + 1) / 2;
    const int64_t items = zp_n * yp_n;
    for (int64_t item = (int64_t)blockIdx.x * kAdj2Warps + warp; item < items;
         item += (int64_t)gridDim.x * kAdj2Warps) {
        const int64_t Yp = item % yp_n, Zp = item / yp_n;
        TW wz[2][3], wy[2][3];
        if (HZ) {
            kt_pair<TW>(Zp, m0, k0, wz);
        } else {
            wz[0][0] = wz[0][2] = wz[1][0] = wz[1][1] = wz[1][2] = TW(0);
            wz[0][1] = TW(1);
        }
        kt_pair<TW>(Yp, m1, k1, wy);
        // coarse rows (Zp-1+a, Yp-1+b), present when inside the coarse grid
        for (int64_t X = lane; X < m2; X += 32) {
            TW acc[2][2] = {{TW(0), TW(0)}, {TW(0), TW(0)}};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int64_t Iz = HZ ? Zp - 1 + a : 0;
                if (HZ ? (Iz < 0 || Iz >= m0) : a != 1) continue;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int64_t Iy = Yp - 1 + b;
                    if (Iy < 0 || Iy >= m1) continue;
                    const TW v = Zc[(Iz * m1 + Iy) * m2 + X];
#pragma unroll
                    for (int pz = 0; pz < 2; ++pz)
#pragma unroll
                        for (int py = 0; py < 2; ++py) acc[pz][py] += wz[pz][a] * wy[py][b] * v;
                }
            }
#pragma unroll
            for (int pz = 0; pz < 2; ++pz)
#pragma unroll
                for (int py = 0; py < 2; ++py) R[(pz * 2 + py) * m2 + X] = acc[pz][py];
        }
        __syncwarp();
        for (int64_t x = lane; x < n2; x += 32) {
            // dim-2 stencil weights of fine column x over R
            const int64_t Xh = x >> 1;
            TW wx[3];
            if (!(x & 1)) {
                wx[0] = (Xh - 1 >= 0) ? k2[5 * (Xh - 1) + 4] : TW(0);
                wx[1] = k2[5 * Xh + 2];
                wx[2] = (Xh + 1 < m2) ? k2[5 * (Xh + 1)] : TW(0);
            } else {
                wx[0] = TW(0);
                wx[1] = k2[5 * Xh + 3];
                wx[2] = (Xh + 1 < m2) ? k2[5 * (Xh + 1) + 1] : TW(0);
            }
#pragma unroll
            for (int pz = 0; pz < 2; ++pz) {
                const int64_t z = HZ ? 2 * Zp + pz : 0;
                if (HZ ? z >= n0 : pz != 0) continue;
#pragma unroll
                for (int py = 0; py < 2; ++py) {
                    const int64_t y = 2 * Yp + py;
                    if (y >= n1) continue;
                    if (!((x & 1) || py || pz)) continue;  // a node of N_{l-1}
                    const TW *r = R + (pz * 2 + py) * m2;
                    TW g = wx[1] * r[Xh];
                    if (Xh - 1 >= 0) g += wx[0] * r[Xh - 1];
                    if (Xh + 1 < m2) g += wx[2] * r[Xh + 1];
                    T *pa = A + (z * n1 + y) * n2 + x;
                    const TW av = static_cast<TW>(*pa);
                    *pa = static_cast<T>(p.sign > 0 ? av + g : av - g);
                }
            }
        }
        __syncwarp();
    }
}

// k_adj_even2 (2D/3D): the same map as k_adj_even, separably.  The sum of
// Pi^T over the 3 x 3 x 3 fine box of a coarse node reads only nodes of
// N_l \ N_{l-1} besides the node itself, whose weight is 1, so
//   s = sum_{a,b,c} wz_a wy_b wx_c A(box) - A(node).
// A warp takes one coarse row (Zc, Yc): per fine column it folds the nine
// fine rows (2Zc-1.., 2Yc-1..) with wz wy (two fine columns per lane,
// 2X and 2X+1), and the dim-2 weights combine column 2X-1 (the previous
// lane's, carried across chunks by lane 31), 2X and 2X+1.
template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(32 * kAdj2Warps) k_adj_even2(AdjParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ B = static_cast<const TW *>(p.Z);  // compact base, or null: A itself
    const T *w0 = static_cast<const T *>(p.w0);
    const T *w1 = static_cast<const T *>(p.w1);
    const T *w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t items = m0 * m1;
    for (int64_t item = (int64_t)blockIdx.x * kAdj2Warps + warp; item < items;
         item += (int64_t)gridDim.x * kAdj2Warps) {
        const int64_t Yc = item % m1, Zc = item / m1;
        // weights of the fine planes / rows 2E-1, 2E, 2E+1 of coarse index E
        TW wz[3], wy[3];
        if (HZ) {
            wz[0] = (Zc >= 1) ? static_cast<TW>(w0[2 * (2 * Zc - 1) + 1]) : TW(0);
            wz[1] = TW(1);
            wz[2] = (Zc <= m0 - 2) ? static_cast<TW>(w0[2 * (2 * Zc + 1)]) : TW(0);
        } else {
            wz[0] = wz[2] = TW(0);
            wz[1] = TW(1);
        }
        wy[0] = (Yc >= 1) ? static_cast<TW>(w1[2 * (2 * Yc - 1) + 1]) : TW(0);
        wy[1] = TW(1);
        wy[2] = (Yc <= m1 - 2) ? static_cast<TW>(w1[2 * (2 * Yc + 1)]) : TW(0);
        const int64_t ze = HZ ? 2 * Zc : 0, ye = 2 * Yc;
        TW carry = TW(0);  // folded value of fine column 2 X0 - 1
        for (int64_t X0 = 0; X0 < m2; X0 += 32) {
            const int64_t X = X0 + lane;
            const bool v0 = X < m2, v1 = X + 1 < m2;  // fine columns 2X, 2X+1
            TW r0 = TW(0), r1 = TW(0), self = TW(0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (wz[a] == TW(0)) continue;
                const int64_t z = ze - 1 + a;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (wy[b] == TW(0)) continue;
                    const int64_t y = ye - 1 + b;
                    const T *row = A + (z * n1 + y) * n2 + 2 * X;
                    const TW wab = wz[a] * wy[b];
                    const TW a0 = v0 ? static_cast<TW>(row[0]) : TW(0);
                    const TW a1 = v1 ? static_cast<TW>(row[1]) : TW(0);
                    r0 += wab * a0;
                    r1 += wab * a1;
                    if (a == 1 && b == 1) self = a0;
                }
            }
            TW rm = __shfl_up_sync(0xffffffffu, r1, 1);  // fine column 2X - 1
            if (lane == 0) rm = carry;
            carry = __shfl_sync(0xffffffffu, r1, 31);
            if (v0) {
                const TW wr = (X >= 1) ? static_cast<TW>(w2[2 * (2 * X - 1) + 1]) : TW(0);
                const TW wl = v1 ? static_cast<TW>(w2[2 * (2 * X + 1)]) : TW(0);
                const TW s2 = wr * rm + r0 + wl * r1 - self;
                T *pe = A + (ze * n1 + ye) * n2 + 2 * X;
                const TW base = B ? B[(Zc * m1 + Yc) * m2 + X] : self;
                *pe = static_cast<T>(p.sign > 0 ? base + s2 : base - s2);
            }
        }
    }
}

}  // namespace mg
