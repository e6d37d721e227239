// rowchunk.cuh -- level kernels over rows in coalesced 16-byte words.
//
// A warp takes one segment of a row: Q sub-segments of W = 32 E fine
// columns (E elements per 16-byte word).  In sub-segment q lane L owns the
// E columns W q + E L .. W q + E L + E - 1 (its "canonical" columns), and
// the lane of the row's last segment also the row's final column.  Every
// row of a level array with 2^k + 1 columns starts at a different offset A
// inside a 16-byte word (n2 is odd); with n1 = n2 = 1 mod 4 the offset of
// row (z, y) is (z + y) mod E, so within one step of a kernel every row's
// offset is a compile-time constant once the step's first is known: each
// step is compiled per offset and selected at run time.
//
// Loads: in sub-segment q lane L reads aligned word 32 q + L of the segment,
// so a warp reads 512 consecutive bytes per instruction; the A + 1 values
// its canonical window needs beyond its word come from lane L + 1 by a
// rotating shuffle (lane 31 from lane 0's next word), the left halo of the
// restriction from lane L - 1.  Stores write the same aligned words whole,
// their first A values taken from lane L - 1; only the segment's first and
// last words are written in parts.  Compact coarse rows (F, V) move in pairs
// of coarse values per lane, shifted by one lane value where the row starts
// at an odd offset.
//
// k_rc_sweep<MODE_DEC> (decomposition, Section II-A-1): the coefficients
//   u - Pi_{l-1} u on N_l \ N_{l-1}, in place; coarse nodes unchanged.
// k_rc_sweep<MODE_REC> (recomposition, Section II-A): N_{l-1} nodes take the
//   corrected coarse values V, every other node its coefficient plus the
//   multilinear interpolant of V.
// Both stream the planes of a chunk for one coarse row (fine rows 2Y, 2Y+1):
// per coarse plane Z the interpolant I2 of its two rows (dim 2 on the even
// row, then dim 1 on the odd row), kept in registers for the odd plane
// 2Z + 1 after it (dim 0).
//
// k_rc_restrict (both directions, Section III-A-2):
//   F = (K_0 (x) K_1 (x) K_2) C,  C = A on N_l \ N_{l-1}, 0 on N_{l-1}
//   V = A restricted to N_{l-1}
// for a block of TY coarse rows of one segment, streaming the planes of
// a chunk: per fine row the dim-2 stencil of the lane's coarse columns (two
// per word of 4-byte elements, one of 8-byte ones), the dim-1 stencil into
// register accumulators, the dim-0 stencil into rolling accumulators over
// the plane pairs (2Z - 1, 2Z).  With XS (a row is one segment) the solve of
// M_{l-1} along dim 2 runs on each finished row of F before it is stored:
// the row is handed to lanes in contiguous chunks through a per-warp
// shared-memory row, each lane runs the Thomas recurrences of the tabulated
// LU factors over its chunk from a zero carry, the chunk maps are composed
// across the warp by a shuffle scan, and each chunk re-runs from its true
// carry (Section III-A-3).
#pragma once

#include "common.cuh"
#include "params.h"

namespace mg {

constexpr unsigned kRcFull = 0xffffffffu;

template <int N>
struct IC {
    static constexpr int value = N;
};

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(IC<I>{});
        static_for<I + 1, N>(f);
    }
}

template <typename T>
struct VecE {
    static constexpr int value = 16 / (int)sizeof(T);
};

template <typename T>
__device__ __forceinline__ void ld16(const T *p, T *o)
{
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x;
        o[1] = v.y;
    }
}

template <typename T>
__device__ __forceinline__ void st16(T *p, const T *v)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
}

// two consecutive elements at an address aligned to their joint size
template <typename T>
__device__ __forceinline__ void ld_pair(const T *p, T &a, T &b)
{
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        a = v.x;
        b = v.y;
    }
}

template <typename T>
__device__ __forceinline__ void st_pair(T *p, T a, T b)
{
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    else *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}

// value of lane L + 1, lane 31 taking lane 0's `nxt` (the next sub-segment)
template <typename T>
__device__ __forceinline__ T from_right(T cur, T nxt, int L)
{
    return __shfl_sync(kRcFull, (L == 0) ? nxt : cur, (L + 1) & 31);
}

// value of lane L - 1, lane 0 taking lane 31's `prv` (the previous sub-segment)
template <typename T>
__device__ __forceinline__ T from_left(T cur, T prv, int L)
{
    return __shfl_sync(kRcFull, (L == 31) ? prv : cur, (L + 31) & 31);
}

// ---- per-warp ring of row copies in shared memory
// One commit group of cp.async copies per row position of a warp's fixed
// sequence of rows, issued D positions ahead of their use.  For a field row
// segment lane L copies the aligned words 32 q + L (lane 0 also the word
// after the segment), for a compact row its pairs of coarse values; it later
// reads back exactly the words it copied, so the lanes need no barrier.

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// bytes of a slot: a field row segment (the word before it, its Q W
// columns as words, the word after) or a compact row of TW (WC Q + 2
// values), a 16-byte multiple
template <typename T, typename TW, int Q>
struct RingSlot {
    static constexpr int E = VecE<T>::value, W = 32 * E, NC = E / 2, WC = 32 * NC;
    static constexpr int FIELD_B = (W * Q + 2 * E) * (int)sizeof(T);
    static constexpr int COARSE_B = (WC * Q + 2) * (int)sizeof(TW);
    static constexpr int BYTES = ((FIELD_B > COARSE_B ? FIELD_B : COARSE_B) + 15) / 16 * 16;
};

// Copy the aligned words of the row segment whose first column is seg (word
// offset a): word w of the segment goes to slot word w + 1; lane L copies
// words 32 q + L, lane 0 also the word after the segment and, when
// `before`, the word before it.
template <typename T, int Q>
__device__ __forceinline__ void ring_copy_row(T *slot, const T *seg, int a, int L, bool before)
{
    constexpr int E = VecE<T>::value, W = 32 * E;
    const T *g = seg - a;
#pragma unroll
    for (int q = 0; q < Q; ++q) cp_async16(slot + W * q + E * L + E, g + W * q + E * L);
    if (L == 0) {
        cp_async16(slot + W * Q + E, g + W * Q);
        if (before) cp_async16(slot, g - E);
    }
}

// Canonical windows of a row segment from its slot (every lane's copies
// complete and visible: after the warp's barrier): v[q][H + i] = seg[W q +
// E L + i], i = -H .. E, A = word offset of the segment.  The lane reads its
// own word and its neighbours' from the slot.  Left-halo values of
// sub-segment 0 of lane 0 are 0 at a row start (!left).
template <typename T, int Q, int H, int A>
__device__ __forceinline__ void rw_slot(const T *slot, int L, bool left, T (&v)[Q][H + VecE<T>::value + 1])
{
    constexpr int E = VecE<T>::value, W = 32 * E;
    static_assert(A >= 0 && A < E, "word offset");
    // canonical i is element (i + A) mod E of slot word (own + 1) + floor((i + A) / E)
    constexpr int DLO = (A - H >= 0) ? 0 : -((H - A + E - 1) / E);
    constexpr int DHI = 1;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        T w[DHI - DLO + 1][E];
#pragma unroll
        for (int d = DLO; d <= DHI; ++d) ld16(slot + W * q + E * (L + 1 + d), w[d - DLO]);
#pragma unroll
        for (int i = -H; i <= E; ++i) {
            const int r = i + A;
            const int d = (r >= 0) ? r / E : -((-r + E - 1) / E);
            const int e = r - d * E;
            T x = w[d - DLO][e];
            if (i < 0 && q == 0 && L == 0 && !left) x = T(0);
            v[q][H + i] = x;
        }
    }
}

// Copy a compact row window (pairs of coarse values from crow - par, pair
// index 32 q + L; lane 0 also pair 32 Q), or single values for NC = 1.
template <typename TW, int Q, int NC>
__device__ __forceinline__ void ring_copy_crow(TW *slot, const TW *crow, int par, int L)
{
    constexpr int WC = 32 * NC;
    if constexpr (NC == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) cp_async_elem(slot + WC * q + L, crow + WC * q + L, true);
        if (L == 0) cp_async_elem(slot + WC * Q, crow + WC * Q, true);
    } else {
        const TW *g = crow - par;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if constexpr (sizeof(TW) == 4) cp_async8(slot + WC * q + 2 * L, g + WC * q + 2 * L);
            else cp_async16(slot + WC * q + 2 * L, g + WC * q + 2 * L);
        }
        if (L == 0) {
            if constexpr (sizeof(TW) == 4) cp_async8(slot + WC * Q, g + WC * Q);
            else cp_async16(slot + WC * Q, g + WC * Q);
        }
    }
}

// Compact row window from its slot (after the warp's barrier):
// v[q][j] = crow[WC q + NC L + j], j = 0 .. NC; par = (offset of crow) mod 2.
template <typename TW, int Q, int NC>
__device__ __forceinline__ void c_slot(const TW *slot, int L, int par, TW (&v)[Q][NC + 1])
{
    constexpr int WC = 32 * NC;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if constexpr (NC == 1) {
            v[q][0] = slot[WC * q + L];
            v[q][1] = slot[WC * q + L + 1];
        } else {
            TW a, b, a2, b2;
            ld_pair(slot + WC * q + 2 * L, a, b);
            ld_pair(slot + WC * q + 2 * L + 2, a2, b2);
            if (par == 0) {
                v[q][0] = a;
                v[q][1] = b;
                v[q][2] = a2;
            } else {  // pairs (2L - 1, 2L)
                v[q][0] = b;
                v[q][1] = a2;
                v[q][2] = b2;
            }
        }
    }
}

// Stores o[q][i] at seg[W q + E L + i], i < E, and o[Q-1][E] at seg[W Q]
// when `extra` (the row's final column, lane 31 of its last segment).
template <typename T, int Q, int A>
__device__ __forceinline__ void rw_store(T *seg, int L, const T (&o)[Q][VecE<T>::value + 1], bool extra)
{
    constexpr int E = VecE<T>::value, W = 32 * E;
    static_assert(A >= 0 && A < E, "word offset");
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        T wv[E];
#pragma unroll
        for (int p = 0; p < E; ++p) {
            if (p >= A) wv[p] = o[q][p - A];
            else wv[p] = from_left(o[q][E + p - A], o[q > 0 ? q - 1 : 0][E + p - A], L);
        }
        T *w0 = seg + W * q + E * L - A;
        if (A > 0 && q == 0 && L == 0) {
#pragma unroll
            for (int p = A; p < E; ++p) w0[p] = wv[p];
        } else {
            st16(w0, wv);
        }
    }
    if (L == 31) {
#pragma unroll
        for (int i = E - A; i < E; ++i) seg[W * Q - E + i] = o[Q - 1][i];
        if (extra) seg[W * Q] = o[Q - 1][E];
    }
}

// Compact coarse row of a segment (crow = its first coarse column; WC = 32 NC
// coarse columns per sub-segment): lane L's values o[q][j] at crow[WC q + NC
// L + j], and ox at crow[WC Q] when `extra`.  par = (element offset of crow)
// mod 2 (NC = 2: pairs start at even offsets).
template <typename TW, int Q, int NC>
__device__ __forceinline__ void c_store(TW *crow, int L, const TW (&o)[Q][NC], TW ox, bool extra, int par)
{
    constexpr int WC = 32 * NC;
    if constexpr (NC == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) crow[WC * q + L] = o[q][0];
    } else {
        static_assert(NC == 2, "one or two coarse values per lane");
        if (par == 0) {
#pragma unroll
            for (int q = 0; q < Q; ++q) st_pair(crow + WC * q + 2 * L, o[q][0], o[q][1]);
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const TW prev = from_left(o[q][1], o[q > 0 ? q - 1 : 0][1], L);
                if (q == 0 && L == 0) crow[0] = o[0][0];
                else st_pair(crow + WC * q + 2 * L - 1, prev, o[q][0]);
            }
            if (L == 31) crow[WC * Q - 1] = o[Q - 1][1];
        }
    }
    if (extra) crow[WC * Q] = ox;
}

// Multilinear interpolation along dim 2 of a canonical window e (even
// columns exact): X[i] = e[i] for even i, wl e[i-1] + wr e[i+1] for odd i.
template <typename T, int Q, bool WU>
__device__ __forceinline__ void x_interp(const T (&e)[Q][VecE<T>::value + 1], const T (&wl)[Q][VecE<T>::value / 2],
                                         const T (&wr)[Q][VecE<T>::value / 2], T (&X)[Q][VecE<T>::value + 1])
{
    constexpr int E = VecE<T>::value;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int i = 0; i <= E; ++i) {
            if (i & 1) X[q][i] = WU ? lerp2(T(0.5), e[q][i - 1], T(0.5), e[q][i + 1])
                                    : lerp2(wl[q][i / 2], e[q][i - 1], wr[q][i / 2], e[q][i + 1]);
            else X[q][i] = e[q][i];
        }
}

// The same from a compact coarse window (coarse j = canonical fine 2 j).
template <typename T, typename TW, int Q, bool WU>
__device__ __forceinline__ void x_interp_c(const TW (&v)[Q][VecE<T>::value / 2 + 1],
                                           const T (&wl)[Q][VecE<T>::value / 2], const T (&wr)[Q][VecE<T>::value / 2],
                                           T (&X)[Q][VecE<T>::value + 1])
{
    constexpr int E = VecE<T>::value;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int i = 0; i <= E; ++i) {
            if (i & 1) {
                const T a = static_cast<T>(v[q][i / 2]), b = static_cast<T>(v[q][i / 2 + 1]);
                X[q][i] = WU ? lerp2(T(0.5), a, T(0.5), b) : lerp2(wl[q][i / 2], a, wr[q][i / 2], b);
            } else {
                X[q][i] = static_cast<T>(v[q][i / 2]);
            }
        }
}

// Rows a sweep step reads, in order of use (RPS per coarse plane Z):
//   DEC: (2Z, 2Y), (2Z, 2Y+1), (2Z, 2Y+2), (2Z-1, 2Y), (2Z-1, 2Y+1)
//   REC: V(Z, Y), V(Z, Y+1), (2Z, 2Y), (2Z, 2Y+1), (2Z-1, 2Y), (2Z-1, 2Y+1)
template <int MODE>
struct SweepSeq {
    static constexpr int RPS = MODE == MODE_DEC ? 5 : 6;
    static constexpr int D = 2 * RPS - 1;  // prefetch distance (row positions)
    static constexpr int NSLOT = D + 1;
};

template <typename T, typename TW, int Q, int MODE>
inline size_t rc_sweep_smem()
{
    return (size_t)kRcWarps * SweepSeq<MODE>::NSLOT * RingSlot<T, TW, Q>::BYTES;
}

template <typename T, typename TW, int Q, bool HZ, int MODE, bool WU>
__global__ void __launch_bounds__(32 * kRcWarps) k_rc_sweep(RcParams p)
{
    constexpr bool DEC = (MODE == MODE_DEC);
    constexpr int E = VecE<T>::value, W = 32 * E, NC = E / 2;
    constexpr int RPS = SweepSeq<MODE>::RPS, D = SweepSeq<MODE>::D, NSLOT = SweepSeq<MODE>::NSLOT;
    constexpr int SB = RingSlot<T, TW, Q>::BYTES;
    using Row = T[Q][E + 1];
    extern __shared__ __align__(16) unsigned char rc_smem[];
    unsigned char *ring = rc_smem + (size_t)(threadIdx.x >> 5) * NSLOT * SB;
    T *__restrict__ A = static_cast<T *>(p.A);
    const TW *__restrict__ V = static_cast<const TW *>(p.V);
    const T *__restrict__ w0 = static_cast<const T *>(p.w0);
    const T *__restrict__ w1 = static_cast<const T *>(p.w1);
    const T *__restrict__ w2 = static_cast<const T *>(p.w2);
    const int L = threadIdx.x & 31;
    const int n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2, S = p.S;
    const int64_t plane = (int64_t)n1 * n2;
    pdl_wait();

    for (int item = blockIdx.x * kRcWarps + (threadIdx.x >> 5); item < p.nitems; item += gridDim.x * kRcWarps) {
        const int s = item % S;
        const int rest = item / S;
        const int Y = rest % m1;
        const int c = rest / m1;
        const bool extra = (L == 31) && (s == S - 1);
        const bool two = Y + 1 < m1;  // the odd row 2Y+1 (and the next even row) exist
        const int col0 = W * Q * s, ccol0 = (W / 2) * Q * s;
        const int Z0 = HZ ? c * p.zchunk : 0;
        const int Z1 = HZ ? min(Z0 + p.zchunk, m0 - 1) : 0;

        // issue the copies of the next row position (positions in order of
        // use; an empty group past the end): coarse plane iz, row kind ik
        int iz = Z0, ik = 0, islot = 0;
        auto issue = [&]() {
            if (iz <= Z1) {
                void *slot = ring + islot * SB;
                int kf = ik;  // field row kind: 0 = (2Z, 2Y) .. 4 = (2Z-1, 2Y+1)
                if constexpr (!DEC) {
                    if (ik < 2) {
                        if (ik == 0 || two)
                            ring_copy_crow<TW, Q, NC>(static_cast<TW *>(slot), V + ((int64_t)iz * m1 + Y + ik) * m2 + ccol0,
                                                      (iz + Y + ik) & 1, L);
                        kf = -1;
                    } else {
                        kf = (ik == 2) ? 0 : (ik == 3 ? 1 : ik - 1);
                    }
                }
                if (kf >= 0) {
                    // kf = 0, 1, 2: rows 2Y, 2Y+1, 2Y+2 of plane 2Z; 3, 4: rows 2Y, 2Y+1 of plane 2Z-1
                    const bool oddp = kf >= 3;
                    const int z = oddp ? 2 * iz - 1 : 2 * iz;
                    const int y = 2 * Y + (oddp ? kf - 3 : kf);
                    const bool ok = (!oddp || (HZ && iz > Z0)) && (y == 2 * Y || two);
                    if (ok)
                        ring_copy_row<T, Q>(static_cast<T *>(slot), A + ((int64_t)z * n1 + y) * n2 + col0, (z + y) % E,
                                            L, false);
                }
            }
            cp_async_commit();
            if (++ik == RPS) {
                ik = 0;
                ++iz;
            }
            if (++islot == NSLOT) islot = 0;
        };
        // wait for row position i and make every lane's copies visible; its
        // slot stays valid until the next take (whose copies refill the
        // slot of position i - 1 + NSLOT, the one after it in the ring)
        int tslot = 0;
        auto take = [&]() -> const unsigned char * {
            __syncwarp();  // every lane has read the slot that issue() refills
            issue();
            cp_async_wait<D>();
            __syncwarp();
            const unsigned char *r = ring + tslot * SB;
            if (++tslot == NSLOT) tslot = 0;
            return r;
        };
#pragma unroll 1
        for (int j = 0; j < D; ++j) issue();

        T wl[Q][NC], wr[Q][NC];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                if constexpr (WU) {
                    wl[q][j] = wr[q][j] = T(0.5);
                } else {
                    const int col = col0 + W * q + E * L + 2 * j + 1;
                    wl[q][j] = w2[2 * col];
                    wr[q][j] = w2[2 * col + 1];
                }
            }
        const T wyl = two ? w1[2 * (2 * Y + 1)] : T(0), wyr = two ? w1[2 * (2 * Y + 1) + 1] : T(0);

        T I2p[2][Q][E + 1], I2c[2][Q][E + 1];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int i = 0; i <= E; ++i) I2p[r][q][i] = I2c[r][q][i] = T(0);

        for (int Z = Z0; Z <= Z1; ++Z) {
            const bool own_even = !HZ || Z < Z1 || Z == m0 - 1;
            const bool odd = HZ && Z > Z0;  // the odd plane 2Z - 1 is this item's
            T *segA = A + ((int64_t)(2 * Z) * n1 + 2 * Y) * n2 + col0;  // even plane 2Z, row 2Y
            T wzl = T(0), wzr = T(0);
            if (odd) {
                wzl = w0[2 * (2 * Z - 1)];
                wzr = w0[2 * (2 * Z - 1) + 1];
            }
            const int par = (Z + Y) & 1;  // offset of row (2Z, 2Y) is 2 par mod E
            auto step = [&](auto PC) {
                constexpr int A0 = (2 * decltype(PC)::value) % E;
                Row cA, cB, X0, XH;
                if constexpr (DEC) {
                    Row eH;
                    rw_slot<T, Q, 0, A0>(reinterpret_cast<const T *>(take()), L, false, cA);
                    rw_slot<T, Q, 0, (A0 + 1) % E>(reinterpret_cast<const T *>(take()), L, false, cB);
                    rw_slot<T, Q, 0, (A0 + 2) % E>(reinterpret_cast<const T *>(take()), L, false, eH);
                    x_interp<T, Q, WU>(cA, wl, wr, X0);
                    x_interp<T, Q, WU>(eH, wl, wr, XH);
                } else {
                    TW vA[Q][NC + 1], vH[Q][NC + 1];
                    c_slot<TW, Q, NC>(reinterpret_cast<const TW *>(take()), L, par, vA);
                    c_slot<TW, Q, NC>(reinterpret_cast<const TW *>(take()), L, par ^ 1, vH);
                    rw_slot<T, Q, 0, A0>(reinterpret_cast<const T *>(take()), L, false, cA);
                    rw_slot<T, Q, 0, (A0 + 1) % E>(reinterpret_cast<const T *>(take()), L, false, cB);
                    x_interp_c<T, TW, Q, WU>(vA, wl, wr, X0);
                    x_interp_c<T, TW, Q, WU>(vH, wl, wr, XH);
                }
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int i = 0; i <= E; ++i) {
                        I2c[0][q][i] = X0[q][i];
                        I2c[1][q][i] = lerp2(wyl, X0[q][i], wyr, XH[q][i]);
                    }
                if (own_even) {
                    Row out;
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int i = 0; i <= E; ++i) {
                            if constexpr (DEC) out[q][i] = (i & 1) ? sub_rn(cA[q][i], X0[q][i]) : cA[q][i];
                            else out[q][i] = (i & 1) ? add_rn(cA[q][i], X0[q][i]) : X0[q][i];
                        }
                    rw_store<T, Q, A0>(segA, L, out, extra);
                    if (two) {
#pragma unroll
                        for (int q = 0; q < Q; ++q)
#pragma unroll
                            for (int i = 0; i <= E; ++i)
                                out[q][i] = DEC ? sub_rn(cB[q][i], I2c[1][q][i]) : add_rn(cB[q][i], I2c[1][q][i]);
                        rw_store<T, Q, (A0 + 1) % E>(segA + n2, L, out, extra);
                    }
                }
                // the odd plane 2Z - 1 (its positions are taken in any case;
                // each slot is read before the next take)
                Row oA, oB;
                const T *sO = reinterpret_cast<const T *>(take());
                if (odd) rw_slot<T, Q, 0, (A0 + E - 1) % E>(sO, L, false, oA);
                const T *sO2 = reinterpret_cast<const T *>(take());
                if (odd) rw_slot<T, Q, 0, A0>(sO2, L, false, oB);
                if (odd) {
                    T *segO = segA - plane;  // plane 2Z - 1, row 2Y
                    Row out;
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int i = 0; i <= E; ++i) {
                            const T I = lerp2(wzl, I2p[0][q][i], wzr, I2c[0][q][i]);
                            out[q][i] = DEC ? sub_rn(oA[q][i], I) : add_rn(oA[q][i], I);
                        }
                    rw_store<T, Q, (A0 + E - 1) % E>(segO, L, out, extra);
                    if (two) {
#pragma unroll
                        for (int q = 0; q < Q; ++q)
#pragma unroll
                            for (int i = 0; i <= E; ++i) {
                                const T I = lerp2(wzl, I2p[1][q][i], wzr, I2c[1][q][i]);
                                out[q][i] = DEC ? sub_rn(oB[q][i], I) : add_rn(oB[q][i], I);
                            }
                        rw_store<T, Q, A0>(segO + n2, L, out, extra);
                    }
                }
            };
            if (par) step(IC<1>{});
            else step(IC<0>{});
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int i = 0; i <= E; ++i) I2p[r][q][i] = I2c[r][q][i];
        }
        cp_async_wait<0>();  // the ring is reused by the next item
    }
}

// Solve of M_{l-1} along a row held by the warp in contiguous chunks: lane L
// nodes C2 L .. C2 L + C2 - 1 in f[0 .. C2), lane 31 also the row's final
// node in f[C2] (the row has 32 C2 + 1 nodes).  sfac: factors (a, inv, q)
// of the lane's nodes in shared memory at [(t C2 + k) 32 + L]; xa, xi: a
// and inv of the final node (its q is 0).
template <typename TW, int C2>
__device__ __forceinline__ void rc_xsolve(TW (&f)[C2 + 1], const TW *sfac, TW xa, TW xi, int L)
{
    const bool last = (L == 31);
    // forward y_i = f_i - a_i y_{i-1}: the chunk as the map y_in -> y_out = Y + P y_in
    TW y = TW(0), P = TW(1);
#pragma unroll
    for (int k = 0; k < C2; ++k) {
        const TW a = sfac[k * 32 + L];
        y = f[k] - a * y;
        P = -a * P;
    }
    if (last) {
        y = f[C2] - xa * y;
        P = -xa * P;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const TW Yp = __shfl_up_sync(kRcFull, y, d), Pp = __shfl_up_sync(kRcFull, P, d);
        if (L >= d) {
            y = y + P * Yp;
            P = P * Pp;
        }
    }
    TW carry = __shfl_up_sync(kRcFull, y, 1);
    if (L == 0) carry = TW(0);
    y = carry;
#pragma unroll
    for (int k = 0; k < C2; ++k) {
        y = f[k] - sfac[k * 32 + L] * y;
        f[k] = y;
    }
    if (last) f[C2] = f[C2] - xa * y;
    // backward z_i = inv_i y_i - q_i z_{i+1}, chunk maps composed from the right
    TW z = TW(0);
    P = TW(1);
    if (last) z = xi * f[C2];
#pragma unroll
    for (int k = C2 - 1; k >= 0; --k) {
        const TW q = sfac[(2 * C2 + k) * 32 + L];
        z = sfac[(C2 + k) * 32 + L] * f[k] - q * z;
        P = -q * P;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const TW Zn = __shfl_down_sync(kRcFull, z, d), Pn = __shfl_down_sync(kRcFull, P, d);
        if (L + d < 32) {
            z = z + P * Zn;
            P = P * Pn;
        }
    }
    carry = __shfl_down_sync(kRcFull, z, 1);
    if (last) carry = TW(0);
    z = carry;
    if (last) {
        z = xi * f[C2];
        f[C2] = z;
    }
#pragma unroll
    for (int k = C2 - 1; k >= 0; --k) {
        z = sfac[(C2 + k) * 32 + L] * f[k] - sfac[(2 * C2 + k) * 32 + L] * z;
        f[k] = z;
    }
}

// prefetch distance of the restriction's ring (row positions)
constexpr int kRcRestrictD = 7;

// Shared memory of k_rc_restrict, in bytes: the warps' rings (kRcRestrictD
// + 1 field-row slots each); with XS the factors of the chunk nodes (3 C2 32
// of TW) and one row of 32 C2 + 1 nodes per warp (TW); for non-uniform K_2
// the rows of every segment's lane nodes (5 C2 32 S of T); C2 = coarse nodes
// per lane and segment.
template <typename T, typename TW, int Q>
inline size_t rc_restrict_smem(int S, bool ku, bool xs)
{
    constexpr size_t C2 = (size_t)(VecE<T>::value / 2) * Q;
    size_t b = (size_t)kRcWarps * (kRcRestrictD + 1) * RingSlot<T, TW, Q>::BYTES;
    if (xs) b += (3 * C2 * 32 + (size_t)kRcWarps * (32 * C2 + 4)) * sizeof(TW);
    b = (b + 15) / 16 * 16;
    if (!ku) b += 5 * C2 * 32 * (size_t)S * sizeof(T);
    return b;
}

template <typename T, typename TW, int Q, bool HZ, bool KU, bool XS, int TY>
__global__ void __launch_bounds__(32 * kRcWarps) k_rc_restrict(RcParams p)
{
    pdl_wait();
    constexpr int E = VecE<T>::value, W = 32 * E, NC = E / 2, WC = 32 * NC;
    constexpr int C2 = NC * Q;      // coarse nodes per lane and segment
    constexpr int NR = 2 * TY + 3;  // fine rows feeding TY coarse rows
    constexpr int PPZ = HZ ? 2 * NR : NR;  // row positions per coarse plane (odd plane, even plane)
    constexpr int D = kRcRestrictD, NSLOT = D + 1;
    constexpr int SB = RingSlot<T, TW, Q>::BYTES;
    extern __shared__ __align__(16) unsigned char rc_smem[];
    unsigned char *ring = rc_smem + (size_t)(threadIdx.x >> 5) * NSLOT * SB;
    TW *sfac = reinterpret_cast<TW *>(rc_smem + (size_t)kRcWarps * NSLOT * SB);
    TW *srow = sfac + 3 * C2 * 32 + (threadIdx.x >> 5) * (32 * C2 + 4);
    T *sk2 = reinterpret_cast<T *>(
        rc_smem + (((size_t)kRcWarps * NSLOT * SB +
                    (XS ? (3 * C2 * 32 + kRcWarps * (32 * C2 + 4)) * sizeof(TW) : 0)) + 15) / 16 * 16);
    const T *__restrict__ A = static_cast<const T *>(p.A);
    TW *__restrict__ F = static_cast<TW *>(p.F);
    TW *__restrict__ V = static_cast<TW *>(p.V);
    const T *__restrict__ k0 = static_cast<const T *>(p.k0);
    const T *__restrict__ k1 = static_cast<const T *>(p.k1);
    const T *__restrict__ k2 = static_cast<const T *>(p.k2);
    const TW *__restrict__ fx = static_cast<const TW *>(p.fx);
    const int L = threadIdx.x & 31;
    const int n1 = p.n1, n2 = p.n2, m0 = p.m0, m1 = p.m1, m2 = p.m2, S = p.S;
    const int64_t plane = (int64_t)n1 * n2, cplane = (int64_t)m1 * m2;

    // per-block tables: the LU factors of a row's nodes in contiguous lane
    // chunks (XS: a row is one segment), and for non-uniform grids the K_2
    // rows of the lanes' coarse nodes
    if constexpr (XS) {
        for (int e = threadIdx.x; e < 3 * C2 * 32; e += blockDim.x) {
            const int t = e / (C2 * 32), k = (e / 32) % C2, l = e % 32;
            sfac[e] = fx[3 * (C2 * l + k) + t];
        }
    }
    if constexpr (!KU) {
        // [t][q][j][s][L]: node WC (Q s + q) + NC L + j
        for (int e = threadIdx.x; e < 5 * C2 * 32 * S; e += blockDim.x) {
            const int l = e % 32, s = (e / 32) % S, j = (e / (32 * S)) % NC, q = (e / (32 * S * NC)) % Q;
            const int t = e / (32 * S * NC * Q);
            sk2[e] = k2[5 * (WC * (Q * s + q) + NC * l + j) + t];
        }
    }
    __syncthreads();
    TW xa = TW(0), xi = TW(0);
    if constexpr (XS) {
        xa = fx[3 * (m2 - 1)];
        xi = fx[3 * (m2 - 1) + 1];
    }

    for (int item = blockIdx.x * kRcWarps + (threadIdx.x >> 5); item < p.nitems; item += gridDim.x * kRcWarps) {
        const int s = item % S;
        const int rest = item / S;
        const int b = rest % p.nb;
        const int c = rest / p.nb;
        const int yown = TY * b;
        const int Y0 = min(yown, m1 - TY);  // a last block ends at the final coarse row
        const bool extra = (L == 31) && (s == S - 1);
        const int col0 = W * Q * s, ccol0 = WC * Q * s;
        const int Zs = HZ ? c * p.zchunk : 0;
        const int Ze = HZ ? (c == p.nzc - 1 ? m0 : Zs + p.zchunk) : 1;
        const int Zfirst = (HZ && Zs > 0) ? Zs - 1 : Zs;
        const int Zlast = HZ ? min(Ze, m0 - 1) : 0;

        // row positions in order of use: per coarse plane Zfirst.. the odd
        // plane's NR rows 2 Y0 - 2 .. 2 Y0 + 2 TY (3D), then the even
        // plane's; issue() copies the next one (coarse plane iz, kind ik)
        int iz = Zfirst, ik = 0, islot = 0;
        auto issue = [&]() {
            const bool oddp = HZ && ik < NR;
            const int r = oddp ? ik : ik - (HZ ? NR : 0);
            const int y = 2 * Y0 - 2 + r;
            const bool ok = iz <= Zlast && y >= 0 && y < n1 && (!oddp || (iz >= 1 && iz >= Zs));
            if (ok) {
                const int z = oddp ? 2 * iz - 1 : (HZ ? 2 * iz : 0);
                ring_copy_row<T, Q>(reinterpret_cast<T *>(ring + islot * SB), A + ((int64_t)z * n1 + y) * n2 + col0,
                                    (z + y) % E, L, s > 0);
            }
            cp_async_commit();
            if (++ik == PPZ) {
                ik = 0;
                ++iz;
            }
            if (++islot == NSLOT) islot = 0;
        };
        int tslot = 0;
        auto take = [&]() -> const T * {
            __syncwarp();  // every lane has read the slot that issue() refills
            issue();
            cp_async_wait<D>();
            __syncwarp();
            const T *r = reinterpret_cast<const T *>(ring + tslot * SB);
            if (++tslot == NSLOT) tslot = 0;
            return r;
        };
#pragma unroll 1
        for (int j = 0; j < D; ++j) issue();

        // K_2 rows: interior rows shared (KU); the lane's first node of
        // sub-segment 0 (the grid's first at L = 0 of segment 0) and the
        // final node separately
        T kc[5], kb0[5], kbx[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            kc[t] = KU ? k2[5 + t] : T(0);
            kb0[t] = KU ? k2[5 * (ccol0 + NC * L) + t] : T(0);
            kbx[t] = extra ? k2[5 * (m2 - 1) + t] : T(0);
        }
        auto kx = [&](int q, int j, int t) -> T {
            if constexpr (KU) return (q == 0 && j == 0) ? kb0[t] : kc[t];
            else return sk2[(((t * Q + q) * NC + j) * S + s) * 32 + L];
        };

        T acc[3][TY][Q][NC], accx[3][TY];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int j = 0; j < TY; ++j) {
                accx[u][j] = T(0);
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int k = 0; k < NC; ++k) acc[u][j][q][k] = T(0);
            }

        // F rows Zo of the block (own rows only), solved along dim 2 with XS
        auto store_f = [&](int Zo) {
#pragma unroll
            for (int j = 0; j < TY; ++j) {
                if (Y0 + j < yown) continue;
                TW o[Q][NC];
                TW ox = static_cast<TW>(accx[0][j]);
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int k = 0; k < NC; ++k) o[q][k] = static_cast<TW>(acc[0][j][q][k]);
                if constexpr (XS) {
                    // to contiguous lane chunks through the warp's row, solve, back
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int k = 0; k < NC; ++k) srow[WC * q + NC * L + k] = o[q][k];
                    if (L == 31) srow[32 * C2] = ox;
                    __syncwarp();
                    TW f[C2 + 1];
#pragma unroll
                    for (int k = 0; k < C2; ++k) f[k] = srow[C2 * L + k];
                    f[C2] = (L == 31) ? srow[32 * C2] : TW(0);
                    __syncwarp();
                    rc_xsolve<TW, C2>(f, sfac, xa, xi, L);
#pragma unroll
                    for (int k = 0; k < C2; ++k) srow[C2 * L + k] = f[k];
                    if (L == 31) srow[32 * C2] = f[C2];
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int k = 0; k < NC; ++k) o[q][k] = srow[WC * q + NC * L + k];
                    if (L == 31) ox = srow[32 * C2];
                    __syncwarp();
                }
                TW *frow = F + (int64_t)Zo * cplane + (int64_t)(Y0 + j) * m2 + ccol0;
                c_store<TW, Q, NC>(frow, L, o, ox, extra, (Zo + Y0 + j) & 1);
            }
        };

        for (int Z = Zfirst; Z <= Zlast; ++Z) {
            const bool has_odd = HZ && Z >= 1 && Z >= Zs;
            const bool own_even = Z >= Zs && Z < Ze;
            // dim-2 and dim-1 stencils of fine plane `pl` into g; AP = word
            // offset of its row 2 Y0 - 2; EVEN: an even plane (its even rows
            // hold coarse nodes, C = 0 there, and those are gathered into V)
            auto plane_pass = [&](auto APC, auto EVC, const T *pl, int Zv, T (&g)[TY][Q][NC], T (&gx)[TY]) {
                constexpr int AP = decltype(APC)::value;
                constexpr bool EVEN = decltype(EVC)::value != 0;
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    gx[j] = T(0);
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int k = 0; k < NC; ++k) g[j][q][k] = T(0);
                }
                static_for<0, NR>([&](auto RC) {
                    constexpr int r = decltype(RC)::value;
                    const int y = 2 * Y0 - 2 + r;
                    const T *slot = take();
                    if (y < 0 || y >= n1) return;
                    T v[Q][E + 3];
                    rw_slot<T, Q, 2, (AP + r) % E>(slot, L, s > 0, v);
                    constexpr bool MASK = EVEN && (r % 2 == 0);
                    T h[Q][NC], hx;
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int k = 0; k < NC; ++k) {
                            // taps at canonical columns 2k - 2 .. 2k + 2 = v[q][2k .. 2k + 4]
                            if constexpr (MASK) {
                                h[q][k] = fma_rn(kx(q, k, 1), v[q][2 * k + 1], mul_rn(kx(q, k, 3), v[q][2 * k + 3]));
                            } else {
                                T t = mul_rn(kx(q, k, 0), v[q][2 * k]);
                                t = fma_rn(kx(q, k, 1), v[q][2 * k + 1], t);
                                t = fma_rn(kx(q, k, 2), v[q][2 * k + 2], t);
                                t = fma_rn(kx(q, k, 3), v[q][2 * k + 3], t);
                                h[q][k] = fma_rn(kx(q, k, 4), v[q][2 * k + 4], t);
                            }
                        }
                    // the final node (canonical column E of the last sub-segment): taps 0 .. 2
                    if constexpr (MASK) {
                        hx = mul_rn(kbx[1], v[Q - 1][E + 1]);
                    } else {
                        T t = mul_rn(kbx[0], v[Q - 1][E]);
                        t = fma_rn(kbx[1], v[Q - 1][E + 1], t);
                        hx = fma_rn(kbx[2], v[Q - 1][E + 2], t);
                    }
                    if constexpr (EVEN && r % 2 == 0) {
                        // coarse row Y0 - 1 + r / 2 of coarse plane Zv into V
                        const int Yr = Y0 - 1 + r / 2;
                        if (own_even && Yr >= yown && Yr < Y0 + TY) {
                            TW o[Q][NC];
#pragma unroll
                            for (int q = 0; q < Q; ++q)
#pragma unroll
                                for (int k = 0; k < NC; ++k) o[q][k] = static_cast<TW>(v[q][2 + 2 * k]);
                            TW *vrow = V + (int64_t)Zv * cplane + (int64_t)Yr * m2 + ccol0;
                            c_store<TW, Q, NC>(vrow, L, o, static_cast<TW>(v[Q - 1][2 + E]), extra, (Zv + Yr) & 1);
                        }
                    }
                    // fine row 2 Y0 - 2 + r feeds coarse row Y0 + j with tap r - 2 j
                    static_for<0, TY>([&](auto JC) {
                        constexpr int j = decltype(JC)::value;
                        constexpr int t = r - 2 * j;
                        if constexpr (t >= 0 && t <= 4) {
                            const T ky = __ldg(k1 + 5 * (Y0 + j) + t);
#pragma unroll
                            for (int q = 0; q < Q; ++q)
#pragma unroll
                                for (int k = 0; k < NC; ++k) g[j][q][k] = fma_rn(ky, h[q][k], g[j][q][k]);
                            gx[j] = fma_rn(ky, hx, gx[j]);
                        }
                    });
                });
            };
            auto step = [&](auto AC) {
                constexpr int A0 = decltype(AC)::value;  // offset of row (2Z, 2 Y0 - 2)
                T g[TY][Q][NC], gx[TY];
                if constexpr (HZ) {
                    if (!has_odd) {
#pragma unroll 1
                        for (int r = 0; r < NR; ++r) take();  // the positions of the missing plane
                    } else {  // plane 2Z - 1: tap 3 of Z - 1, tap 1 of Z
                        plane_pass(IC<(A0 + E - 1) % E>{}, IC<0>{}, A + (int64_t)(2 * Z - 1) * plane + col0, Z, g, gx);
                        const T kzP3 = __ldg(k0 + 5 * (Z - 1) + 3), kzC1 = __ldg(k0 + 5 * Z + 1);
#pragma unroll
                        for (int j = 0; j < TY; ++j) {
                            accx[0][j] = fma_rn(kzP3, gx[j], accx[0][j]);
                            accx[1][j] = fma_rn(kzC1, gx[j], accx[1][j]);
#pragma unroll
                            for (int q = 0; q < Q; ++q)
#pragma unroll
                                for (int k = 0; k < NC; ++k) {
                                    acc[0][j][q][k] = fma_rn(kzP3, g[j][q][k], acc[0][j][q][k]);
                                    acc[1][j][q][k] = fma_rn(kzC1, g[j][q][k], acc[1][j][q][k]);
                                }
                        }
                    }
                }
                // even plane 2Z: tap 4 of Z - 1, tap 2 of Z, tap 0 of Z + 1
                plane_pass(IC<A0>{}, IC<1>{}, A + (int64_t)(HZ ? 2 * Z : 0) * plane + col0, HZ ? Z : 0, g, gx);
                if constexpr (HZ) {
                    const T kzP4 = (Z >= 1) ? __ldg(k0 + 5 * (Z - 1) + 4) : T(0);
                    const T kzC2 = __ldg(k0 + 5 * Z + 2);
                    const T kzN0 = (Z + 1 < m0) ? __ldg(k0 + 5 * (Z + 1)) : T(0);
#pragma unroll
                    for (int j = 0; j < TY; ++j) {
                        accx[0][j] = fma_rn(kzP4, gx[j], accx[0][j]);
                        accx[1][j] = fma_rn(kzC2, gx[j], accx[1][j]);
                        accx[2][j] = mul_rn(kzN0, gx[j]);
#pragma unroll
                        for (int q = 0; q < Q; ++q)
#pragma unroll
                            for (int k = 0; k < NC; ++k) {
                                acc[0][j][q][k] = fma_rn(kzP4, g[j][q][k], acc[0][j][q][k]);
                                acc[1][j][q][k] = fma_rn(kzC2, g[j][q][k], acc[1][j][q][k]);
                                acc[2][j][q][k] = mul_rn(kzN0, g[j][q][k]);
                            }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < TY; ++j) {
                        accx[0][j] = gx[j];
#pragma unroll
                        for (int q = 0; q < Q; ++q)
#pragma unroll
                            for (int k = 0; k < NC; ++k) acc[0][j][q][k] = g[j][q][k];
                    }
                }
            };
            // row (2Z, 2 Y0 - 2) starts at offset 2 (Z + Y0 - 1) mod E
            if ((Z + Y0 + 1) & 1) step(IC<2 % E>{});
            else step(IC<0>{});
            if constexpr (HZ) {
                // F(Z - 1) is complete once the planes up to 2Z are in
                if (Z - 1 >= Zs && Z - 1 < Ze) store_f(Z - 1);
#pragma unroll
                for (int j = 0; j < TY; ++j) {
                    accx[0][j] = accx[1][j];
                    accx[1][j] = accx[2][j];
#pragma unroll
                    for (int q = 0; q < Q; ++q)
#pragma unroll
                        for (int k = 0; k < NC; ++k) {
                            acc[0][j][q][k] = acc[1][j][q][k];
                            acc[1][j][q][k] = acc[2][j][q][k];
                        }
                }
            }
        }
        // the last coarse plane of the grid has no contributions beyond it
        if constexpr (HZ) {
            if (Zlast == m0 - 1 && m0 - 1 >= Zs && m0 - 1 < Ze) store_f(m0 - 1);
        } else {
            store_f(0);
        }
        cp_async_wait<0>();  // the ring is reused by the next item
    }
}

}  // namespace mg
