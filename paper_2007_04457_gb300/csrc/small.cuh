// small.cuh -- every remaining level of a small level array in one block.
//
// The coarse end of the hierarchy (arrays of a few thousand to some tens of
// thousands of nodes) costs little arithmetic but a dozen dependent launches
// per level.  k_small loads such an array into shared memory once and runs
// all of its levels there -- the same four steps per level as the tiled path
// (Section II-A, Eq. 1-2; Section III-A):
//   decomposition, level stride s = 1, 2, 4, ...:
//     C = U - Pi U_coarse on the nodes of N_l \ N_{l-1} (written in place),
//     F = (K_0 (x) K_1 (x) K_2) C  (5-point rows K = P^T M_l per dimension),
//     M_{l-1} z = F along every dimension (Thomas, LU factors tabulated),
//     U_coarse += z;
//   recomposition, coarsest level first: F from the stored coefficients, the
//     same solves, U_coarse -= z, then U = C + Pi U_coarse on N_l \ N_{l-1}.
// Level l works on the nodes of the array whose indices are multiples of s in
// every active dimension, so the array ends in the in-place layout of the
// whole transform.  Arithmetic is in TW; the global array has type T.
//
// Shared memory (elements of TW): the array U, then G (dims 1 and 2 reduced,
// all fine planes of the first level), F (the first level's coarse grid), H
// (dim 2 reduced, a chunk of fine planes at a time; hcap elements) and the
// tables of every level.
#pragma once

#include "common.cuh"
#include "small_params.h"

namespace mg {

constexpr int kSmallThreads = 1024;

template <typename TW>
struct SmallLevel {
    int nf[3], nc[3];    // fine / coarse node counts (inactive dims: 1)
    int act[3];          // 1 for an active dimension
    int st[3];           // array strides of one fine index step
    const TW *w[3], *k[3], *fac[3];
};

// floor(e / d) for 0 <= e < 2^17 and 1 <= d < 2^17, from rcp = 1.0f / d
// (IEEE-rounded): (e + 1/2) / d is at least 1/(2d) away from an integer and
// the float product errs by less than 2^-6 / d, so truncation is exact.
__device__ __forceinline__ int small_div(int e, float rcp)
{
    return __float2int_rz((static_cast<float>(e) + 0.5f) * rcp);
}

// U = U + sgn * Pi U_coarse at every node of N_l \ N_{l-1} (sgn = -1: the
// coefficients of a decomposition; +1: the values of a recomposition).
// Nested linear interpolation, dim 2 first; a dimension with an even index
// takes weights (1, 0) and a zero offset, which reproduces the corner value
// exactly, so every node runs the same instructions.  Reads only coarse
// nodes, which the pass does not write.
template <typename TW>
__device__ void small_interp_pass(TW *U, const SmallLevel<TW> &L, TW sgn)
{
    const int nf1 = L.nf[1], nf2 = L.nf[2];
    const float r1 = 1.0f / (float)nf1, r2 = 1.0f / (float)nf2;
    const int total = L.nf[0] * nf1 * nf2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int row = small_div(e, r2), i2 = e - row * nf2;
        const int i0 = small_div(row, r1), i1 = row - i0 * nf1;
        const int o0 = L.act[0] & i0, o1 = L.act[1] & i1, o2 = L.act[2] & i2 & 1;
        if (!((o0 | o1 | o2) & 1)) continue;
        const int q0 = o0 & 1, q1 = o1 & 1;
        const TW wl0 = q0 ? L.w[0][2 * i0] : TW(1), wr0 = q0 ? L.w[0][2 * i0 + 1] : TW(0);
        const TW wl1 = q1 ? L.w[1][2 * i1] : TW(1), wr1 = q1 ? L.w[1][2 * i1 + 1] : TW(0);
        const TW wl2 = o2 ? L.w[2][2 * i2] : TW(1), wr2 = o2 ? L.w[2][2 * i2 + 1] : TW(0);
        const int b = (i0 - q0) * L.st[0] + (i1 - q1) * L.st[1] + (i2 - o2) * L.st[2];
        const int d0 = 2 * q0 * L.st[0], d1 = 2 * q1 * L.st[1], d2 = 2 * o2 * L.st[2];
        const TW x00 = wl2 * U[b] + wr2 * U[b + d2];
        const TW x01 = wl2 * U[b + d1] + wr2 * U[b + d1 + d2];
        const TW x10 = wl2 * U[b + d0] + wr2 * U[b + d0 + d2];
        const TW x11 = wl2 * U[b + d0 + d1] + wr2 * U[b + d0 + d1 + d2];
        const TW y0 = wl1 * x00 + wr1 * x01, y1 = wl1 * x10 + wr1 * x11;
        const TW I = wl0 * y0 + wr0 * y1;
        TW &u = U[i0 * L.st[0] + i1 * L.st[1] + i2 * L.st[2]];
        u = u + sgn * I;
    }
}

// F = (K_0 (x) K_1 (x) K_2) C with C = U on N_l \ N_{l-1} and 0 on N_{l-1}:
// dim 2 into H (a chunk of fine planes at a time), dim 1 into G (every fine
// plane), dim 0 into F.
template <typename TW>
__device__ void small_load_vector(const TW *U, TW *G, TW *F, TW *H, int hcap, const SmallLevel<TW> &L)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nf0 = L.nf[0], nf1 = L.nf[1], nf2 = L.nf[2];
    const int nc0 = L.nc[0], nc1 = L.nc[1], nc2 = L.nc[2];
    const float rc1 = 1.0f / (float)nc1, rc2 = 1.0f / (float)nc2, rf1 = 1.0f / (float)nf1;
    const int chunk = max(1, min(nf0, hcap / (nf1 * nc2)));
    for (int c0 = 0; c0 < nf0; c0 += chunk) {
        const int np = min(chunk, nf0 - c0);
        // H(p, i1, X) = sum_c K_2[X][c] C(c0 + p, i1, 2X - 2 + c)
        for (int e = tid; e < np * nf1 * nc2; e += nt) {
            const int r = small_div(e, rc2), X = e - r * nc2;
            const int p = small_div(r, rf1), i1 = r - p * nf1, i0 = c0 + p;
            const bool row_odd = ((L.act[0] & i0) | (L.act[1] & i1)) & 1;
            const TW *u = U + i0 * L.st[0] + i1 * L.st[1];
            TW h = TW(0);
            if (L.act[2]) {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const int i2 = 2 * X - 2 + c;
                    const bool use = i2 >= 0 && i2 < nf2 && (row_odd || (c & 1));
                    if (use) h += L.k[2][5 * X + c] * u[i2 * L.st[2]];
                }
            } else if (row_odd) {
                h = u[0];
            }
            H[e] = h;
        }
        __syncthreads();
        // G(i0, Y, X) = sum_b K_1[Y][b] H(p, 2Y - 2 + b, X)
        for (int e = tid; e < np * nc1 * nc2; e += nt) {
            const int r = small_div(e, rc2), X = e - r * nc2;
            const int p = small_div(r, rc1), Y = r - p * nc1;
            const TW *h = H + p * nf1 * nc2 + X;
            TW v = TW(0);
            if (L.act[1]) {
#pragma unroll
                for (int b = 0; b < 5; ++b) {
                    const int i1 = 2 * Y - 2 + b;
                    if (i1 >= 0 && i1 < nf1) v += L.k[1][5 * Y + b] * h[i1 * nc2];
                }
            } else {
                v = h[0];
            }
            G[c0 * nc1 * nc2 + e] = v;
        }
        __syncthreads();
    }
    // F(Z, Y, X) = sum_a K_0[Z][a] G(2Z - 2 + a, Y, X)
    const int plane = nc1 * nc2;
    const float rpl = 1.0f / (float)plane;
    for (int e = tid; e < nc0 * plane; e += nt) {
        const int Z = small_div(e, rpl), yx = e - Z * plane;
        TW f = TW(0);
        if (L.act[0]) {
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const int i0 = 2 * Z - 2 + a;
                if (i0 >= 0 && i0 < nf0) f += L.k[0][5 * Z + a] * G[i0 * plane + yx];
            }
        } else {
            f = G[yx];
        }
        F[e] = f;
    }
    __syncthreads();
}

// M z = f along one line of m nodes at stride s in shared memory, in place
// (forward elimination with the multipliers a_i, back substitution with
// 1/pivot and the scaled super-diagonal), a few nodes at a time so that the
// loads of a group are in flight together.
template <typename TW>
__device__ __forceinline__ void line_solve_smem(TW *f, int s, int m, const TW *fac)
{
    constexpr int K = sizeof(TW) == 4 ? 8 : 4;
    TW t = TW(0);
    for (int b = 0; b < m; b += K) {
        TW y[K], a[K];
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (b + u < m) {
                y[u] = f[(b + u) * s];
                a[u] = fac[3 * (b + u)];
            }
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (b + u < m) {
                t = y[u] - a[u] * t;
                f[(b + u) * s] = t;
            }
    }
    t = TW(0);
    for (int b = m - 1; b >= 0; b -= K) {
        TW y[K], iv[K], q[K];
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (b - u >= 0) {
                y[u] = f[(b - u) * s];
                iv[u] = fac[3 * (b - u) + 1];
                q[u] = fac[3 * (b - u) + 2];
            }
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (b - u >= 0) {
                t = iv[u] * y[u] - q[u] * t;
                f[(b - u) * s] = t;
            }
    }
}

// M_{l-1} z = F along every active dimension, in place, one thread per line.
template <typename TW>
__device__ void small_solves(TW *F, const SmallLevel<TW> &L)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nc[3] = {L.nc[0], L.nc[1], L.nc[2]};
    for (int k = 2; k >= 0; --k) {
        if (!L.act[k]) continue;
        const int m = nc[k];
        const int inner = (k == 2) ? 1 : (k == 1 ? nc[2] : nc[1] * nc[2]);
        const int nlines = nc[0] * nc[1] * nc[2] / m;
        const TW *fac = L.fac[k];
        for (int line = tid; line < nlines; line += nt)
            line_solve_smem<TW>(F + (line / inner) * (inner * m) + line % inner, inner, m, fac);
        __syncthreads();
    }
}

// Every level of the array p.A in shared memory `smem` (small_elems + hcap
// + small_tab_elems elements of TW), by the calling block.
template <typename T, typename TW, int MODE>
__device__ void small_run(const SmallParams &p, unsigned char *smem_raw)
{
    TW *U = reinterpret_cast<TW *>(smem_raw);
    const int n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
    const int N = n0 * n1 * n2;
    const int m0 = (n0 > 1) ? (n0 - 1) / 2 + 1 : 1;
    const int m1 = (n1 > 1) ? (n1 - 1) / 2 + 1 : 1;
    const int m2 = (n2 > 1) ? (n2 - 1) / 2 + 1 : 1;
    TW *G = U + N;
    TW *F = G + n0 * m1 * m2;
    TW *H = F + m0 * m1 * m2;
    TW *Tb = H + p.hcap;  // the tables of every level
    T *A = static_cast<T *>(p.A);
    const int tid = threadIdx.x, nt = blockDim.x;

    // every level's tables (per active dim 2 nf weights, 5 nc stencil
    // entries, 3 nc LU factors) and the array, all copies in flight at once
    {
        int toff = 0;
        for (int i = 0; i < p.nlev; ++i) {
            const int n[3] = {n0, n1, n2};
            for (int d = 0; d < 3; ++d) {
                if (n[d] <= 1) continue;
                const int nf = (n[d] - 1) / (1 << i) + 1, nc = (nf - 1) / 2 + 1;
                const TW *gw = static_cast<const TW *>(p.w[i][d]);
                const TW *gk = static_cast<const TW *>(p.k[i][d]);
                const TW *gf = static_cast<const TW *>(p.fac[i][d]);
                for (int e = tid; e < 2 * nf; e += nt) cp_async_elem<TW>(Tb + toff + e, gw + e, true);
                for (int e = tid; e < 5 * nc; e += nt) cp_async_elem<TW>(Tb + toff + 2 * nf + e, gk + e, true);
                for (int e = tid; e < 3 * nc; e += nt) cp_async_elem<TW>(Tb + toff + 2 * nf + 5 * nc + e, gf + e, true);
                toff += 2 * nf + 8 * nc;
            }
        }
    }
    cp_async_commit();
    for (int e = tid; e < N; e += nt) U[e] = static_cast<TW>(A[e]);
    cp_async_wait<0>();
    __syncthreads();
    int level_toff = 0;
    int toffs[kSmallMaxLevels];
    for (int i = 0; i < p.nlev; ++i) {
        toffs[i] = level_toff;
        const int n[3] = {n0, n1, n2};
        for (int d = 0; d < 3; ++d) {
            if (n[d] <= 1) continue;
            const int nf = (n[d] - 1) / (1 << i) + 1, nc = (nf - 1) / 2 + 1;
            level_toff += 2 * nf + 8 * nc;
        }
    }

    for (int it = 0; it < p.nlev; ++it) {
        const int i = (MODE == MODE_DEC) ? it : p.nlev - 1 - it;
        const int s = 1 << i;
        SmallLevel<TW> L;
        const int n[3] = {n0, n1, n2};
        const int st[3] = {n1 * n2, n2, 1};
        int toff = toffs[i];
        for (int d = 0; d < 3; ++d) {
            L.act[d] = n[d] > 1 ? 1 : 0;
            L.nf[d] = L.act[d] ? (n[d] - 1) / s + 1 : 1;
            L.nc[d] = L.act[d] ? (L.nf[d] - 1) / 2 + 1 : 1;
            L.st[d] = st[d] * s;
            const TW *gw = static_cast<const TW *>(p.w[i][d]);
            const TW *gk = static_cast<const TW *>(p.k[i][d]);
            const TW *gf = static_cast<const TW *>(p.fac[i][d]);
            if (L.act[d]) {
                L.w[d] = Tb + toff;
                L.k[d] = Tb + toff + 2 * L.nf[d];
                L.fac[d] = Tb + toff + 2 * L.nf[d] + 5 * L.nc[d];
                toff += 2 * L.nf[d] + 8 * L.nc[d];
            } else {
                L.w[d] = gw;
                L.k[d] = gk;
                L.fac[d] = gf;
            }
        }

        if constexpr (MODE == MODE_DEC) {
            small_interp_pass<TW>(U, L, TW(-1));
            __syncthreads();
        }
        small_load_vector<TW>(U, G, F, H, p.hcap, L);
        small_solves<TW>(F, L);
        // correction of the coarse nodes (stride 2s; inactive dims have index 0)
        {
            const int nc1 = L.nc[1], nc2 = L.nc[2];
            const float rc1 = 1.0f / (float)nc1, rc2 = 1.0f / (float)nc2;
            for (int e = tid; e < L.nc[0] * nc1 * nc2; e += nt) {
                const int r = small_div(e, rc2), X = e - r * nc2;
                const int Z = small_div(r, rc1), Y = r - Z * nc1;
                TW &u = U[2 * (Z * L.st[0] + Y * L.st[1] + X * L.st[2])];
                if constexpr (MODE == MODE_DEC) u = u + F[e];
                else u = u - F[e];
            }
        }
        __syncthreads();
        if constexpr (MODE == MODE_REC) {
            small_interp_pass<TW>(U, L, TW(1));
            __syncthreads();
        }
    }

    for (int e = tid; e < N; e += nt) A[e] = static_cast<T>(U[e]);
}

// Transposed level maps of every remaining level in shared memory (the
// adjoints of k_small's decomposition and recomposition, Section II-A
// transposed).  In the strided in-place layout the gather of a level's
// coarse nodes into V and their placement back are identities, so per level
// (o = N_l \ N_{l-1}, e = N_{l-1}):
//   decomposition transpose, coarsest level first:
//     F = M_{l-1}^{-1} U(e);  U(o) += K^T F;  U(e) -= Pi^T U(o)
//   recomposition transpose, finest level first:
//     U(e) += Pi^T U(o);  F = M_{l-1}^{-1} U(e);  U(o) -= K^T F
// Shared memory: U, then F (the first level's coarse grid), then the tables.

// F <- U at the coarse nodes of level L (compact).
template <typename TW>
__device__ void small_gather_f(const TW *U, TW *F, const SmallLevel<TW> &L)
{
    const int nc1 = L.nc[1], nc2 = L.nc[2];
    const float rc1 = 1.0f / (float)nc1, rc2 = 1.0f / (float)nc2;
    for (int e = threadIdx.x; e < L.nc[0] * nc1 * nc2; e += blockDim.x) {
        const int r = small_div(e, rc2), X = e - r * nc2;
        const int Z = small_div(r, rc1), Y = r - Z * nc1;
        F[e] = U[2 * (Z * L.st[0] + Y * L.st[1] + X * L.st[2])];
    }
}

// Coarse neighbours of fine index j of a dimension with their K^T weights.
template <typename TW>
__device__ __forceinline__ int small_kt(int j, int m, const TW *k, int (&I)[3], TW (&w)[3])
{
    int c = 0;
    const int I0 = j >> 1;
    if (!(j & 1)) {
        if (I0 - 1 >= 0) { I[c] = I0 - 1; w[c] = k[5 * (I0 - 1) + 4]; ++c; }
        I[c] = I0; w[c] = k[5 * I0 + 2]; ++c;
        if (I0 + 1 < m) { I[c] = I0 + 1; w[c] = k[5 * (I0 + 1)]; ++c; }
    } else {
        I[c] = I0; w[c] = k[5 * I0 + 3]; ++c;
        if (I0 + 1 < m) { I[c] = I0 + 1; w[c] = k[5 * (I0 + 1) + 1]; ++c; }
    }
    return c;
}

// U(o) += sg (K^T F)(o) at every node of N_l \ N_{l-1} of level L.
template <typename TW>
__device__ void small_adj_odd(TW *U, const TW *F, const SmallLevel<TW> &L, TW sg)
{
    const int nf1 = L.nf[1], nf2 = L.nf[2], nc1 = L.nc[1], nc2 = L.nc[2];
    const float r1 = 1.0f / (float)nf1, r2 = 1.0f / (float)nf2;
    for (int e = threadIdx.x; e < L.nf[0] * nf1 * nf2; e += blockDim.x) {
        const int row = small_div(e, r2), i2 = e - row * nf2;
        const int i0 = small_div(row, r1), i1 = row - i0 * nf1;
        if (!(((L.act[0] & i0) | (L.act[1] & i1) | (L.act[2] & i2)) & 1)) continue;  // a node of N_{l-1}
        int I0[3] = {0, 0, 0}, I1[3] = {0, 0, 0}, I2[3] = {0, 0, 0};
        TW w0[3] = {TW(1), TW(0), TW(0)}, w1[3] = {TW(1), TW(0), TW(0)}, w2[3] = {TW(1), TW(0), TW(0)};
        const int c0 = L.act[0] ? small_kt<TW>(i0, L.nc[0], L.k[0], I0, w0) : 1;
        const int c1 = L.act[1] ? small_kt<TW>(i1, nc1, L.k[1], I1, w1) : 1;
        const int c2 = L.act[2] ? small_kt<TW>(i2, nc2, L.k[2], I2, w2) : 1;
        TW g = TW(0);
        for (int a = 0; a < c0; ++a) {
            TW gy = TW(0);
            for (int b = 0; b < c1; ++b) {
                const TW *fr = F + (I0[a] * nc1 + I1[b]) * nc2;
                TW gx = TW(0);
                for (int c = 0; c < c2; ++c) gx += w2[c] * fr[I2[c]];
                gy += w1[b] * gx;
            }
            g += w0[a] * gy;
        }
        U[i0 * L.st[0] + i1 * L.st[1] + i2 * L.st[2]] += sg * g;
    }
}

// Fine neighbours of coarse index E of a dimension with their Pi^T weights.
template <typename TW>
__device__ __forceinline__ int small_pt(int E, int n, const TW *w, int (&j)[3], TW (&wt)[3])
{
    int c = 0;
    const int f = 2 * E;
    if (f - 1 >= 1) { j[c] = f - 1; wt[c] = w[2 * (f - 1) + 1]; ++c; }
    j[c] = f; wt[c] = TW(1); ++c;
    if (f + 1 <= n - 2) { j[c] = f + 1; wt[c] = w[2 * (f + 1)]; ++c; }
    return c;
}

// U(e) += sg (Pi^T U|_o)(e) at every node of N_{l-1} of level L (reads only
// nodes of N_l \ N_{l-1}).
template <typename TW>
__device__ void small_adj_even(TW *U, const SmallLevel<TW> &L, TW sg)
{
    const int nc1 = L.nc[1], nc2 = L.nc[2];
    const float rc1 = 1.0f / (float)nc1, rc2 = 1.0f / (float)nc2;
    for (int e = threadIdx.x; e < L.nc[0] * nc1 * nc2; e += blockDim.x) {
        const int r = small_div(e, rc2), E2 = e - r * nc2;
        const int E0 = small_div(r, rc1), E1 = r - E0 * nc1;
        int j0[3] = {0, 0, 0}, j1[3] = {0, 0, 0}, j2[3] = {0, 0, 0};
        TW w0[3] = {TW(1), TW(0), TW(0)}, w1[3] = {TW(1), TW(0), TW(0)}, w2[3] = {TW(1), TW(0), TW(0)};
        const int c0 = L.act[0] ? small_pt<TW>(E0, L.nf[0], L.w[0], j0, w0) : 1;
        const int c1 = L.act[1] ? small_pt<TW>(E1, L.nf[1], L.w[1], j1, w1) : 1;
        const int c2 = L.act[2] ? small_pt<TW>(E2, L.nf[2], L.w[2], j2, w2) : 1;
        const int f0 = L.act[0] ? 2 * E0 : 0, f1 = L.act[1] ? 2 * E1 : 0, f2 = L.act[2] ? 2 * E2 : 0;
        TW sum = TW(0);
        for (int a = 0; a < c0; ++a)
            for (int b = 0; b < c1; ++b)
                for (int c = 0; c < c2; ++c) {
                    if (j0[a] == f0 && j1[b] == f1 && j2[c] == f2) continue;  // the node itself
                    sum += w0[a] * w1[b] * w2[c] * U[j0[a] * L.st[0] + j1[b] * L.st[1] + j2[c] * L.st[2]];
                }
        U[f0 * L.st[0] + f1 * L.st[1] + f2 * L.st[2]] += sg * sum;
    }
}

// DIR 0: transpose of the decomposition; 1: of the recomposition.
template <typename T, typename TW, int DIR>
__device__ void small_adj_run(const SmallParams &p, unsigned char *smem_raw)
{
    TW *U = reinterpret_cast<TW *>(smem_raw);
    const int n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
    const int N = n0 * n1 * n2;
    const int m0 = (n0 > 1) ? (n0 - 1) / 2 + 1 : 1;
    const int m1 = (n1 > 1) ? (n1 - 1) / 2 + 1 : 1;
    const int m2 = (n2 > 1) ? (n2 - 1) / 2 + 1 : 1;
    TW *F = U + N;
    TW *Tb = F + m0 * m1 * m2;
    T *A = static_cast<T *>(p.A);
    const int tid = threadIdx.x, nt = blockDim.x;
    int toffs[kSmallMaxLevels];
    {
        int toff = 0;
        for (int i = 0; i < p.nlev; ++i) {
            toffs[i] = toff;
            const int n[3] = {n0, n1, n2};
            for (int d = 0; d < 3; ++d) {
                if (n[d] <= 1) continue;
                const int nf = (n[d] - 1) / (1 << i) + 1, nc = (nf - 1) / 2 + 1;
                const TW *gw = static_cast<const TW *>(p.w[i][d]);
                const TW *gk = static_cast<const TW *>(p.k[i][d]);
                const TW *gf = static_cast<const TW *>(p.fac[i][d]);
                for (int e = tid; e < 2 * nf; e += nt) cp_async_elem<TW>(Tb + toff + e, gw + e, true);
                for (int e = tid; e < 5 * nc; e += nt) cp_async_elem<TW>(Tb + toff + 2 * nf + e, gk + e, true);
                for (int e = tid; e < 3 * nc; e += nt) cp_async_elem<TW>(Tb + toff + 2 * nf + 5 * nc + e, gf + e, true);
                toff += 2 * nf + 8 * nc;
            }
        }
    }
    cp_async_commit();
    for (int e = tid; e < N; e += nt) U[e] = static_cast<TW>(A[e]);
    cp_async_wait<0>();
    __syncthreads();

    for (int it = 0; it < p.nlev; ++it) {
        const int i = (DIR == 0) ? p.nlev - 1 - it : it;
        const int s = 1 << i;
        SmallLevel<TW> L;
        const int n[3] = {n0, n1, n2};
        const int st[3] = {n1 * n2, n2, 1};
        int toff = toffs[i];
        for (int d = 0; d < 3; ++d) {
            L.act[d] = n[d] > 1 ? 1 : 0;
            L.nf[d] = L.act[d] ? (n[d] - 1) / s + 1 : 1;
            L.nc[d] = L.act[d] ? (L.nf[d] - 1) / 2 + 1 : 1;
            L.st[d] = st[d] * s;
            if (L.act[d]) {
                L.w[d] = Tb + toff;
                L.k[d] = Tb + toff + 2 * L.nf[d];
                L.fac[d] = Tb + toff + 2 * L.nf[d] + 5 * L.nc[d];
                toff += 2 * L.nf[d] + 8 * L.nc[d];
            } else {
                L.w[d] = L.k[d] = L.fac[d] = Tb;
            }
        }
        if constexpr (DIR == 1) {
            small_adj_even<TW>(U, L, TW(1));
            __syncthreads();
        }
        small_gather_f<TW>(U, F, L);
        __syncthreads();
        small_solves<TW>(F, L);
        small_adj_odd<TW>(U, F, L, DIR == 0 ? TW(1) : TW(-1));
        __syncthreads();
        if constexpr (DIR == 0) {
            small_adj_even<TW>(U, L, TW(-1));
            __syncthreads();
        }
    }

    for (int e = tid; e < N; e += nt) A[e] = static_cast<T>(U[e]);
}

template <typename T, typename TW, int DIR>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_adj(SmallParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    extern __shared__ __align__(16) unsigned char smem_raw[];
    small_adj_run<T, TW, DIR>(p, smem_raw);
}

template <typename T, typename TW, int MODE>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small(SmallParams p)
{
    pdl_wait();  // programmatic dependent launch: the predecessor has finished
    extern __shared__ __align__(16) unsigned char smem_raw[];
    small_run<T, TW, MODE>(p, smem_raw);
}

}  // namespace mg
