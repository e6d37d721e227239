// sweep.cuh -- the element-wise level kernels as warp-tile sweeps.
//
// k_sweep<MODE_DEC> (decomposition, after the coarser levels are done):
//   every node of N_l \ N_{l-1} receives its coefficient u - Pi_{l-1} u
//   (Section II-A-1), the N_{l-1} nodes are rewritten with their own
//   unchanged value (whole sectors are written, and a neighbouring tile that
//   reads them as interpolation corners sees the same bits either way).
// k_sweep<MODE_REC> (recomposition, Section II-A): the N_{l-1} nodes
//   receive the corrected coarse values V, every other node its coefficient
//   plus the multilinear interpolant of V.
//
// The interpolant is evaluated separably, dim 2 first, then dim 1, then dim
// 0, each step an explicitly rounded two-point combination (lerp2), so the
// coefficients are bit-identical to the C the restriction kernel computed.
//
// Work item of one warp: 32 consecutive columns (lane = column) x 8 fine
// rows (1 in 1D) x a chunk of fine planes.  The warp streams the chunk's even planes;
// for each it forms the dim-2 interpolant X of its even rows (odd columns
// from the lane's neighbours by shuffles, even columns exact), the dim-1
// interpolant of its odd rows, and keeps that plane's interpolant I2 in
// registers; the odd plane before it then needs only the two I2 planes
// around it.  A tile reads one halo row (its next even row) and a chunk one
// halo plane (its next even plane); in both only nodes of N_{l-1} are used.
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr int kSweepWarps = 4;  // warps per block

// fine rows per warp item (1 for one-dimensional grids): 8 rows keep the
// registers of 4-byte elements at 80, six blocks (24 warps) per SM
template <int ACT, int ELEM>
struct SweepRows {
    static constexpr int value = (ACT & 2) ? 8 : 1;
};

// 4-byte elements: the next step's loads are issued before this step's
// stores (registers for two steps); resident blocks the registers are sized
// for, as measured at 513^3: 5 (decomposition) and 4 (recomposition) with
// that prefetch, 4 for 8-byte elements without it
template <int ELEM>
struct SweepPipe {
    static constexpr bool value = ELEM == 4;
};
template <int ELEM, int MODE>
struct SweepMinBlocks {
    static constexpr int value = ELEM == 4 ? (MODE == MODE_DEC ? 5 : 4) : 4;
};

template <typename T, typename TW, int ACT, int MODE>
__global__ void __launch_bounds__(32 * kSweepWarps, (SweepMinBlocks<(int)sizeof(T), MODE>::value))
k_sweep(PlaceParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0, HY = (ACT & 2) != 0;
    constexpr bool DEC = (MODE == MODE_DEC);
    constexpr int R = SweepRows<ACT, (int)sizeof(T)>::value;
    constexpr int RE = R / 2 + 1;  // even rows of a tile, with its halo row
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2, m1 = p.m1, m2 = p.m2;
    const int sn2 = (int)n2;  // row stride (a level array row has < 2^31 nodes)
    const int L = threadIdx.x & 31;
    const int64_t warp0 = (int64_t)blockIdx.x * kSweepWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kSweepWarps;
    const int64_t tiles_x = (n2 + 31) / 32;
    const int64_t tiles_y = HY ? (n1 + R - 1) / R : 1;
    const int64_t zc = p.zchunk;
    const int64_t items = tiles_x * tiles_y * p.nzc;

    for (int64_t item = warp0; item < items; item += nwarps) {
        const int64_t tx = item % tiles_x;
        const int64_t rest = item / tiles_x;
        const int64_t ty = rest % tiles_y;
        const int64_t tz = rest / tiles_y;
        const int64_t x = tx * 32 + L;
        const bool xv = x < n2;
        const bool xo = xv && (x & 1);          // odd columns are interior (n2 - 1 is even)
        const T wl2 = xo ? w2[2 * x] : T(1), wr2 = xo ? w2[2 * x + 1] : T(0);
        const int64_t y0 = ty * R;
        const int nrow = (int)min64(R, n1 - y0);           // own rows
        const bool hrow = HY && (y0 + R < n1);              // halo row y0 + R exists
        const int64_t z0 = HZ ? tz * zc : 0;
        const int64_t z1 = HZ ? min64(z0 + zc, n0) : 1;     // own planes [z0, z1)
        const int64_t zlast = (HZ && z1 < n0) ? z1 : z1 - 1;  // even: halo plane or the last plane

        T I2p[R], I2c[R];
#pragma unroll
        for (int r = 0; r < R; ++r) I2p[r] = I2c[r] = T(0);

        // Loads of the step at even plane z (and the odd plane z - 1 before
        // it); with PIPE the next step's loads are issued before this step's
        // stores, which go to other planes.
        auto load_step = [&](int64_t z, T (&ue)[RE], T (&va)[RE], T (&vb)[RE], T (&uo)[R], T (&uz)[R]) {
            const bool own = z < z1;
            const bool odd_plane = HZ && z > z0;
            const T *plane = A + (z * n1 + y0) * n2 + (xv ? x : 0);
            const T *oplane = A + ((odd_plane ? z - 1 : z) * n1 + y0) * n2 + (xv ? x : 0);
#pragma unroll
            for (int e = 0; e < RE; ++e) {
                const int r = 2 * e;
                ue[e] = va[e] = vb[e] = T(0);
                const bool live = (HY || r == 0) && (r < nrow || (r == R && hrow));
                const bool mine = own && r < nrow;
                const T *row = plane + r * sn2;
                if constexpr (DEC) {
                    // outside the tile's own rows and planes only N_{l-1} nodes
                    // (even columns) are read: the others belong to another tile
                    if (live && xv && (mine || !(x & 1))) ue[e] = row[0];
                } else {
                    // V(x/2) for every lane (pairs of lanes share it); the odd
                    // lanes' right neighbour V(x/2 + 1) comes from the next lane,
                    // and lane 31's from one more load
                    if (live) {
                        const TW *vrow = V + ((z >> (HZ ? 1 : 0)) * m1 + ((y0 + r) >> 1)) * m2;
                        if (xv) va[e] = static_cast<T>(vrow[x >> 1]);
                        if (L == 31 && xo) vb[e] = static_cast<T>(vrow[(x >> 1) + 1]);
                    }
                    if (live && mine && xo) ue[e] = row[0];
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                uo[r] = uz[r] = T(0);
                if (r >= nrow) continue;
                if (HY && (r & 1) && own && xv) uo[r] = plane[r * sn2];
                if (odd_plane && xv) uz[r] = oplane[r * sn2];
            }
        };

        constexpr bool PIPE = SweepPipe<(int)sizeof(T)>::value;
        T ue[RE], va[RE], vb[RE], uo[R], uz[R];
        T ue2[RE], va2[RE], vb2[RE], uo2[R], uz2[R];
        if (PIPE) load_step(z0, ue, va, vb, uo, uz);
        for (int64_t z = z0; z <= zlast; z += (HZ ? 2 : 1)) {
            const bool own = z < z1;
            const bool odd_plane = HZ && z > z0;  // the odd plane z - 1 is processed with this one
            T *plane = A + (z * n1 + y0) * n2 + (xv ? x : 0);
            T *oplane = A + ((odd_plane ? z - 1 : z) * n1 + y0) * n2 + (xv ? x : 0);
            const int64_t zn = z + (HZ ? 2 : 1);
            if constexpr (PIPE) {
                if (zn <= zlast) load_step(zn, ue2, va2, vb2, uo2, uz2);
            } else {
                load_step(z, ue, va, vb, uo, uz);
            }
            if constexpr (!DEC) {
#pragma unroll
                for (int e = 0; e < RE; ++e) {
                    const T vn = __shfl_down_sync(0xffffffffu, va[e], 1);
                    if (L != 31) vb[e] = vn;
                }
            }
            // ---- dim-2 interpolant of the even rows
            T Xe[RE];
#pragma unroll
            for (int e = 0; e < RE; ++e) {
                if constexpr (DEC) {
                    T un = __shfl_down_sync(0xffffffffu, ue[e], 1);
                    const T up = __shfl_up_sync(0xffffffffu, ue[e], 1);
                    const int r = 2 * e;
                    const bool live = (HY || r == 0) && (r < nrow || (r == R && hrow));
                    if (L == 31 && xo && live) un = plane[r * sn2 + 1];
                    Xe[e] = xo ? lerp2(wl2, up, wr2, un) : ue[e];
                } else {
                    Xe[e] = xo ? lerp2(wl2, va[e], wr2, vb[e]) : va[e];
                }
            }
            // ---- the plane's interpolant I2 (dim 1 on the odd rows)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (HY && (r & 1) && r < nrow) {
                    const T wyl = w1[2 * (y0 + r)], wyr = w1[2 * (y0 + r) + 1];
                    I2c[r] = lerp2(wyl, Xe[r / 2], wyr, Xe[r / 2 + 1]);
                } else {
                    I2c[r] = Xe[r / 2];
                }
            }
            // ---- stores
            if (own && xv) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r >= nrow) break;
                    T out;
                    if (HY && (r & 1)) {
                        out = DEC ? sub_rn(uo[r], I2c[r]) : add_rn(uo[r], I2c[r]);
                    } else {
                        const T u = ue[r / 2];
                        if constexpr (DEC) out = xo ? sub_rn(u, Xe[r / 2]) : u;
                        else out = xo ? add_rn(u, Xe[r / 2]) : Xe[r / 2];
                    }
                    plane[r * sn2] = out;
                }
            }
            if (odd_plane && xv) {
                const int64_t zo = z - 1;
                const T wzl = w0[2 * zo], wzr = w0[2 * zo + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r >= nrow) break;
                    const T I = lerp2(wzl, I2p[r], wzr, I2c[r]);
                    oplane[r * sn2] = DEC ? sub_rn(uz[r], I) : add_rn(uz[r], I);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) I2p[r] = I2c[r];
            if constexpr (PIPE) {
#pragma unroll
                for (int e = 0; e < RE; ++e) {
                    ue[e] = ue2[e];
                    va[e] = va2[e];
                    vb[e] = vb2[e];
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    uo[r] = uo2[r];
                    uz[r] = uz2[r];
                }
            }
        }
    }
}

// k_sweep2 (recomposition, 2D/3D): as k_sweep<MODE_REC>, with two columns per
// lane.  Warp item: 64 columns (lane L: coarse column X = 32 tx + L, fine
// columns 2X, 2X+1) x R rows x a chunk of planes.  Per even row the lane
// reads V(X) once (the warp's 32 reads are consecutive) and the neighbour
// V(X+1) by shuffle (lane 31: one more read); the interpolants of odd rows
// and of the odd plane before come from registers.  The next step's loads
// are issued before this step's stores.
constexpr bool kSweep2Pipe = true;  // prefetch the next step's loads
constexpr int kSweep2Blocks = 3;     // resident blocks the registers are sized for (4 spills)

template <typename T, typename TW, int ACT>
__global__ void __launch_bounds__(32 * kSweepWarps, kSweep2Blocks) k_sweep2(PlaceParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    constexpr bool HZ = (ACT & 4) != 0;
    constexpr int R = 8;           // fine rows per item
    constexpr int RE = R / 2 + 1;  // even rows with the halo row
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2, m1 = p.m1, m2 = p.m2;
    const int sn2 = (int)n2;
    const int L = threadIdx.x & 31;
    const int64_t warp0 = (int64_t)blockIdx.x * kSweepWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kSweepWarps;
    const int64_t tiles_x = (m2 + 31) / 32;
    const int64_t tiles_y = (n1 + R - 1) / R;
    const int64_t zc = p.zchunk;
    const int64_t items = tiles_x * tiles_y * p.nzc;

    for (int64_t item = warp0; item < items; item += nwarps) {
        const int64_t tx = item % tiles_x;
        const int64_t rest = item / tiles_x;
        const int64_t ty = rest % tiles_y;
        const int64_t tz = rest / tiles_y;
        const int64_t X = tx * 32 + L;
        const bool v0 = X < m2, v1 = X + 1 < m2;  // fine columns 2X, 2X+1 exist
        const int64_t c0 = 2 * X;
        const T wl2 = v1 ? w2[2 * (c0 + 1)] : T(0), wr2 = v1 ? w2[2 * (c0 + 1) + 1] : T(0);
        const int64_t y0 = ty * R;
        const int nrow = (int)min64(R, n1 - y0);
        const bool hrow = y0 + R < n1;
        T wy[R / 2][2];  // weights of the odd rows
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const int64_t y = y0 + 2 * k + 1;
            wy[k][0] = (2 * k + 1 < nrow) ? w1[2 * y] : T(0);
            wy[k][1] = (2 * k + 1 < nrow) ? w1[2 * y + 1] : T(0);
        }
        const int64_t z0 = HZ ? tz * zc : 0;
        const int64_t z1 = HZ ? min64(z0 + zc, n0) : 1;
        const int64_t zlast = (HZ && z1 < n0) ? z1 : z1 - 1;

        // loads of the step at even plane z: V of its even rows (and the
        // right neighbour for lane 31), the coefficients of its own rows and
        // of the odd plane z - 1
        auto load_step = [&](int64_t z, T (&vv)[RE], T (&vr)[RE], T (&ce)[R][2], T (&co)[R][2]) {
            const bool own = z < z1;
            const bool odd_plane = HZ && z > z0;
            const TW *vpl = V + (z >> (HZ ? 1 : 0)) * m1 * m2 + (y0 >> 1) * m2 + X;
            const T *pl = A + (z * n1 + y0) * n2 + c0;
            const T *ol = A + ((odd_plane ? z - 1 : z) * n1 + y0) * n2 + c0;
#pragma unroll
            for (int e = 0; e < RE; ++e) {
                const int r = 2 * e;
                const bool live = r < nrow || (r == R && hrow);
                vv[e] = (live && v0) ? static_cast<T>(vpl[(int64_t)e * m2]) : T(0);
                vr[e] = (live && L == 31 && v1) ? static_cast<T>(vpl[(int64_t)e * m2 + 1]) : T(0);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool mine = own && r < nrow;
                ce[r][0] = (mine && (r & 1) && v0) ? pl[r * sn2] : T(0);
                ce[r][1] = (mine && v1) ? pl[r * sn2 + 1] : T(0);
                const bool om = odd_plane && r < nrow;
                co[r][0] = (om && v0) ? ol[r * sn2] : T(0);
                co[r][1] = (om && v1) ? ol[r * sn2 + 1] : T(0);
            }
        };

        T I2p[R][2], I2c[R][2];
#pragma unroll
        for (int r = 0; r < R; ++r) I2p[r][0] = I2p[r][1] = I2c[r][0] = I2c[r][1] = T(0);
        T vv[RE], vr[RE], ce[R][2], co[R][2];
        T vv2[RE], vr2[RE], ce2[R][2], co2[R][2];
        if (kSweep2Pipe) load_step(z0, vv, vr, ce, co);
        for (int64_t z = z0; z <= zlast; z += (HZ ? 2 : 1)) {
            const bool own = z < z1;
            const bool odd_plane = HZ && z > z0;
            T *pl = A + (z * n1 + y0) * n2 + c0;
            T *ol = A + ((odd_plane ? z - 1 : z) * n1 + y0) * n2 + c0;
            const int64_t zn = z + (HZ ? 2 : 1);
            if constexpr (kSweep2Pipe) {
                if (zn <= zlast) load_step(zn, vv2, vr2, ce2, co2);
            } else {
                load_step(z, vv, vr, ce, co);
            }
            // the plane's interpolant: even rows from V (dim 2), odd rows dim 1
            T Xe[RE][2];
#pragma unroll
            for (int e = 0; e < RE; ++e) {
                T vn = __shfl_down_sync(0xffffffffu, vv[e], 1);
                if (L == 31) vn = vr[e];
                Xe[e][0] = vv[e];
                Xe[e][1] = lerp2(wl2, vv[e], wr2, vn);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r & 1) {
                    const int k = r / 2;
                    I2c[r][0] = lerp2(wy[k][0], Xe[k][0], wy[k][1], Xe[k + 1][0]);
                    I2c[r][1] = lerp2(wy[k][0], Xe[k][1], wy[k][1], Xe[k + 1][1]);
                } else {
                    I2c[r][0] = Xe[r / 2][0];
                    I2c[r][1] = Xe[r / 2][1];
                }
            }
            // stores: the even plane (coarse nodes take V), then the odd one
            if (own) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r >= nrow) break;
                    if (v0) pl[r * sn2] = (r & 1) ? add_rn(ce[r][0], I2c[r][0]) : I2c[r][0];
                    if (v1) pl[r * sn2 + 1] = add_rn(ce[r][1], I2c[r][1]);
                }
            }
            if (odd_plane) {
                const int64_t zo = z - 1;
                const T wzl = w0[2 * zo], wzr = w0[2 * zo + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r >= nrow) break;
                    if (v0) ol[r * sn2] = add_rn(co[r][0], lerp2(wzl, I2p[r][0], wzr, I2c[r][0]));
                    if (v1) ol[r * sn2 + 1] = add_rn(co[r][1], lerp2(wzl, I2p[r][1], wzr, I2c[r][1]));
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                I2p[r][0] = I2c[r][0];
                I2p[r][1] = I2c[r][1];
            }
            if constexpr (kSweep2Pipe) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    ce[r][0] = ce2[r][0];
                    ce[r][1] = ce2[r][1];
                    co[r][0] = co2[r][0];
                    co[r][1] = co2[r][1];
                }
#pragma unroll
                for (int e = 0; e < RE; ++e) {
                    vv[e] = vv2[e];
                    vr[e] = vr2[e];
                }
            }
        }
    }
}

}  // namespace mg
