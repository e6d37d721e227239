// api.cu -- the C ABI of include/mgard.h: plan creation (validation, the
// per-level interpolation / stencil / tridiagonal-factor tables), workspace
// layout and the level loops of decomposition and recomposition
// (Section II-A, Eq. 1-2; Section III-B, program structure).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mgard.h"
#include "launch.cuh"
#include "plan_view.h"
#include "quant.cuh"

using namespace mg;

namespace {

thread_local std::string g_last_error;

mgard_status fail(mgard_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

mgard_status cuda_fail(cudaError_t err, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
    return MGARD_ERR_CUDA;
}

}  // namespace

// Error reporting for the other translation units of the library.
mgard_status mg_fail(mgard_status st, const std::string &msg) { return fail(st, msg); }
mgard_status mg_cuda_fail(cudaError_t err, const char *what) { return cuda_fail(err, what); }

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

// One step of the hierarchy: level l = L - j (fine) -> l - 1 (coarse).
struct mgard_level {
    int64_t n[3];        // level-l node counts (inactive dims = 1)
    int64_t m[3];        // level-(l-1) node counts
    int64_t w_off[3];    // interpolation weight pairs (2 per fine node)
    int64_t k_off[3];    // R*M stencil rows (5 per coarse node)
    int64_t t_off[3];    // tridiagonal factors of M_{l-1} (3 per coarse node)
    int co[3];           // 1: the dim coarsens at this level (0: size 1, or kept with all its nodes)
    size_t v_off, f_off; // workspace offsets of V_j and F_j (bytes)
    int rcfg;            // load-vector tile configuration
    bool rcfg_user;      // set by mgard_plan_tune (else chosen per level)
    int svar;            // warps per line in the solve kernel (0 = automatic)
    int zreq;            // requested coarse planes per restriction item (0 = automatic)
    int zchunk, nzc, tiles_y, tiles_x;
    int rgrid_dec, rgrid_rec;
    int kuni32[3], kuni64[3];  // 1: the interior rows of K (float / double table) are all equal
    int wuni2;           // 1: every odd node of dim 2 has interpolation weights (1/2, 1/2)
    // row-chunk kernels (rowchunk.cuh): used when rc_q[0] > 0; per kernel
    // (sweep, restriction) the sub-segments per segment and segments per row
    int rc_q[2] = {0, 0}, rc_s[2] = {0, 0};
    bool rc_xs = false;          // the restriction also solves along dim 2
    int rc_grid[2] = {0, 0};     // blocks: sweep, restriction
    int rc_zc[2] = {0, 0};       // coarse intervals (sweep) / planes (restriction) per chunk
    int rc_nzc[2] = {0, 0};      // chunk counts
    // slab load-vector kernel (slab.cuh): used when slab_ty > 0
    int slab_ty = 0, slab_ns = 0, slab_sb = 0;  // coarse rows per band, ring slots, slot bytes
    int slab_mb = 0;                            // register variant: blocks per SM (2 or 3)
    int slab_zreq = 0;                          // tune: coarse planes per chunk (0: automatic)
    bool slab_xs = false;                       // the slab kernel also solves along dim 2
    int slab_nb = 0, slab_zc = 0, slab_nzc = 0, slab_grid = 0;
};

struct mgard_plan {
    int ndim;            // squeezed dimension count
    // per-dimension level counts: some dim stops coarsening before the last
    // level; such a plan runs on the persistent kernel (an internal batch of
    // this one field)
    bool per_dim = false;
    mgard_batch *pd_batch = nullptr;
    int act;             // active-dimension mask (ACT_1D / ACT_2D / ACT_3D)
    int64_t n[3];        // finest node counts, leading dims padded with 1
    int L;
    mgard_dtype dtype;
    int device;
    int num_sms;
    size_t elem_user, elem_ws;
    std::vector<mgard_level> lv;
    double *tab64 = nullptr;
    float *tab32 = nullptr;
    bool owns_tables = true;
    size_t ws_bytes = 0;
    int row_grid;
    // levels small_j .. L-1 run in the single-block kernel (small_j = L: none)
    int small_j = 0;
    int small_auto = 0;    // the finest level whose array fits the kernel
    size_t small_smem = 0;
    int small_hcap = 0;
    // the adjoints run levels adj_j .. L-1 in one block (adj_j = L: none): the
    // single-block transposed maps are not separable, so they start only on
    // arrays of at most kAdjSmallNodes nodes
    int adj_j = 0;
    size_t adj_smem = 0;
    // levels coop_j .. L-1 in one cooperative launch (coop_j = L: none):
    // coop_j .. coop_s-1 by the whole grid, coop_s .. L-1 by block 0 in
    // shared memory; coop_auto is the plan's choice, coop_off a tune switch
    int coop_j = 0, coop_auto = 0, coop_s = 0;
    bool coop_off = false;
    int coop_spin = 0;                // barrier poll limit (0: default)
    int rc_off = kRcDefaultOff;       // tune: row-chunk kernels kept out (bit 0 sweeps, bit 1 restriction)
    int rc_zreq = 0;                  // tune: coarse intervals / planes per row-chunk item (0: automatic)
    bool slab_off = false;            // tune: the slab load-vector kernel kept out
    int slab_tyreq = 0, slab_nsreq = 0;  // tune: its rows per band, ring slots (0: automatic)
    int slab_mbreq = 0;               // tune: its register variant, blocks per SM 2 or 3 (0: automatic)
    bool slab_xs_on = false;          // tune: the slab kernel also solves along dim 2 (measured slower)
    int slab_hook = 0;                // tune: test hook (each block's first copy wait runs out)
    unsigned long long slab_wait_ns = 2000000000ull;  // limit of one copy wait
    unsigned *d_status = nullptr;     // device status word of the slab kernel (owned)
    int coop_grid = 0;
    size_t coop_smem = 0;
    int coop_hcap = 0;
    size_t coop_bar_off = 0;
    std::vector<size_t> coop_g_off;   // per grid level: G (n0 x m1 x m2)
    // recomposition from the first coefficient classes: per count D = 1..L of
    // dropped levels (index D - 1) and dim, the table of the weight of every
    // finest node's right N_{L-D} neighbour
    std::vector<std::array<int64_t, 3>> pro_off;
    // kernel timing (measurement support): event pairs around the launches of
    // the prof_levels finest levels
    struct ProfRec {
        int kind, level;
        cudaEvent_t a, b;
    };
    mutable int prof_levels = 0;
    mutable std::vector<ProfRec> prof_pending;
    mutable std::vector<cudaEvent_t> prof_pool;
};

namespace {

int64_t count(const int64_t *n) { return n[0] * n[1] * n[2]; }

// Host construction of one dimension's tables at one level.
//   x: coordinates of the level-l nodes (nf of them).
void build_dim_tables(const std::vector<double> &x, std::vector<double> &tab, int64_t *w_off,
                      int64_t *k_off, int64_t *t_off)
{
    const int64_t nf = (int64_t)x.size();
    const int64_t nc = (nf - 1) / 2 + 1;
    auto h = [&](int64_t i) -> double {  // spacing to the right of fine node i
        return (i >= 0 && i < nf - 1) ? x[i + 1] - x[i] : 0.0;
    };
    // interpolation weights at odd fine nodes: left / right coarse neighbour
    *w_off = (int64_t)tab.size();
    std::vector<double> wl(nf, 0.0), wr(nf, 0.0);
    for (int64_t j = 1; j < nf - 1; j += 2) {
        const double span = x[j + 1] - x[j - 1];
        wl[j] = (x[j + 1] - x[j]) / span;
        wr[j] = (x[j] - x[j - 1]) / span;
    }
    for (int64_t j = 0; j < nf; ++j) {
        tab.push_back(wl[j]);
        tab.push_back(wr[j]);
    }
    // K = P^T M_l restricted to the band: row I covers fine nodes 2I-2 .. 2I+2.
    // M_l (P1 mass matrix scaled by 6): diag 2(h_{i-1}+h_i), off-diagonal h_i.
    auto mass = [&](int64_t r, int64_t c) -> double {
        if (r < 0 || r >= nf || c < 0 || c >= nf) return 0.0;
        if (r == c) return 2.0 * (h(r - 1) + h(r));
        if (c == r + 1) return h(r);
        if (c == r - 1) return h(c);
        return 0.0;
    };
    *k_off = (int64_t)tab.size();
    for (int64_t I = 0; I < nc; ++I) {
        for (int t = 0; t < 5; ++t) {
            const int64_t j = 2 * I - 2 + t;
            double v = 0.0;
            if (j >= 0 && j < nf) {
                v += mass(2 * I, j);                                   // P[2I][I] = 1
                if (2 * I - 1 >= 0) v += wr[2 * I - 1] * mass(2 * I - 1, j);  // P[2I-1][I]
                if (2 * I + 1 < nf) v += wl[2 * I + 1] * mass(2 * I + 1, j);  // P[2I+1][I]
            }
            tab.push_back(v);
        }
    }
    // LU factors of M_{l-1} on the coarse nodes x[0], x[2], ...
    *t_off = (int64_t)tab.size();
    std::vector<double> xc(nc);
    for (int64_t i = 0; i < nc; ++i) xc[i] = x[2 * i];
    auto hc = [&](int64_t i) -> double { return (i >= 0 && i < nc - 1) ? xc[i + 1] - xc[i] : 0.0; };
    double piv_prev = 0.0;
    for (int64_t i = 0; i < nc; ++i) {
        const double d = 2.0 * (hc(i - 1) + hc(i));
        double a = 0.0, piv = d;
        if (i > 0) {
            a = hc(i - 1) / piv_prev;       // multiplier of row i
            piv = d - a * hc(i - 1);
        }
        const double inv = 1.0 / piv;
        const double q = (i < nc - 1) ? hc(i) * inv : 0.0;
        tab.push_back(a);
        tab.push_back(inv);
        tab.push_back(q);
        piv_prev = piv;
    }
}

template <typename T>
const T *tab_ptr(const mgard_plan *P, int64_t off);
template <>
const float *tab_ptr<float>(const mgard_plan *P, int64_t off) { return P->tab32 + off; }
template <>
const double *tab_ptr<double>(const mgard_plan *P, int64_t off) { return P->tab64 + off; }

int act_of(int ndim) { return ndim == 1 ? ACT_1D : (ndim == 2 ? ACT_2D : ACT_3D); }

constexpr int64_t kAdjSmallNodes = 5000;

// First level of the single-block transposed maps: from small_j on, the
// first array of at most kAdjSmallNodes nodes; its shared memory holds the
// array, the first level's coarse grid and the tables of its levels.
void adj_select(mgard_plan *P)
{
    P->adj_j = P->L;
    P->adj_smem = 0;
    for (int j = P->small_j; j < P->L; ++j) {
        const int64_t *nj = (j == 0) ? P->n : P->lv[j - 1].m;
        if (nj[0] * nj[1] * nj[2] > kAdjSmallNodes) continue;
        int64_t m[3];
        for (int k = 0; k < 3; ++k) m[k] = (nj[k] > 1) ? (nj[k] - 1) / 2 + 1 : 1;
        P->adj_j = j;
        P->adj_smem = (size_t)((nj[0] * nj[1] * nj[2] + m[0] * m[1] * m[2] + small_tab_elems(nj, P->L - j)) *
                               (int64_t)P->elem_ws);
        return;
    }
}

enum { KIND_RESTRICT_DEC = 0, KIND_RESTRICT_REC = 1, KIND_SOLVE = 2, KIND_SOLVE_FUSED = 3,
       KIND_PLACE = 4, KIND_INTERP = 5, KIND_PLACE_EVEN = 6, KIND_ADJ = 7, KIND_SMALL = 8,
       KIND_MULTI = 9, KIND_PROLONG = 10 };

cudaEvent_t prof_event(const mgard_plan *P)
{
    if (!P->prof_pool.empty()) {
        cudaEvent_t e = P->prof_pool.back();
        P->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch `fn` on `st`, bracketed by an event pair when level j is profiled.
template <typename Fn>
cudaError_t timed(const mgard_plan *P, int kind, int j, cudaStream_t st, Fn &&fn)
{
    if (j >= P->prof_levels) return fn();
    cudaEvent_t a = prof_event(P), b = prof_event(P);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t err = cudaEventRecord(a, st);
    if (err == cudaSuccess) err = fn();
    if (err == cudaSuccess) err = cudaEventRecord(b, st);
    P->prof_pending.push_back({kind, j, a, b});
    return err;
}

template <typename T, typename TW>
cudaError_t run_restrict_level(const mgard_plan *P, int j, int mode, void *A, char *ws, cudaStream_t st)
{
    const mgard_level &L = P->lv[j];
    RestrictParams p;
    p.A = A;
    p.F = ws + L.f_off;
    p.V = ws + L.v_off;
    p.n0 = L.n[0]; p.n1 = L.n[1]; p.n2 = L.n[2];
    p.m0 = L.m[0]; p.m1 = L.m[1]; p.m2 = L.m[2];
    p.w0 = tab_ptr<T>(P, L.w_off[0]); p.w1 = tab_ptr<T>(P, L.w_off[1]); p.w2 = tab_ptr<T>(P, L.w_off[2]);
    p.k0 = tab_ptr<T>(P, L.k_off[0]); p.k1 = tab_ptr<T>(P, L.k_off[1]); p.k2 = tab_ptr<T>(P, L.k_off[2]);
    p.tiles_y = L.tiles_y;
    p.tiles_x = L.tiles_x;
    p.zchunk = L.zchunk;
    p.nzc = L.nzc;
    p.nitems = L.tiles_y * L.tiles_x * L.nzc;
    p.kuni1 = (sizeof(T) == 4) ? L.kuni32[1] : L.kuni64[1];
    const int grid = (mode == MODE_DEC) ? L.rgrid_dec : L.rgrid_rec;
    return timed(P, mode == MODE_DEC ? KIND_RESTRICT_DEC : KIND_RESTRICT_REC, j, st,
                 [&] { return launch_restrict<T, TW>(P->act, mode, L.rcfg, p, grid, st); });
}

// Solves of M_{l-1} along every active dimension, fastest first; the last
// (slowest) one applies V += z (sign +1), V -= z (sign -1) or leaves z in F
// (sign 0).  With src, the first sweep reads its right-hand sides from src.
template <typename TW>
cudaError_t run_solves(const mgard_plan *P, int j, int sign, char *ws, cudaStream_t st, const void *src = nullptr,
                       int first = 0)
{
    const mgard_level &L = P->lv[j];
    const int nd = P->ndim;
    for (int q = first; q < nd; ++q) {
        const int k = 2 - q;  // internal dim index, fastest first
        SolveParams sp;
        sp.F = ws + L.f_off;
        sp.V = ws + L.v_off;
        sp.fac = tab_ptr<TW>(P, L.t_off[k]);
        sp.m = (int)L.m[k];
        int64_t inner = 1;
        for (int r = k + 1; r < 3; ++r) inner *= L.m[r];
        sp.inner = inner;
        sp.stride = inner;
        sp.nlines = count(L.m) / L.m[k];
        sp.chunk = 0;
        sp.nw = 0;
        sp.lpb = 32;
        sp.vmode = (q == nd - 1) ? (sign > 0 ? 1 : (sign < 0 ? 2 : 0)) : 0;
        sp.src = (q == first) ? src : nullptr;  // the first sweep may read its right-hand sides elsewhere
        cudaError_t err = timed(P, sp.vmode ? KIND_SOLVE_FUSED : KIND_SOLVE, j, st,
                                [&] { return launch_solve<TW>(sp, L.svar, P->num_sms, st); });
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

template <typename T>
PlaceParams place_params(const mgard_plan *P, int j, void *A, char *ws)
{
    const mgard_level &L = P->lv[j];
    PlaceParams p;
    p.A = A;
    p.V = ws + L.v_off;
    p.n0 = L.n[0]; p.n1 = L.n[1]; p.n2 = L.n[2];
    p.m0 = L.m[0]; p.m1 = L.m[1]; p.m2 = L.m[2];
    p.w0 = tab_ptr<T>(P, L.w_off[0]); p.w1 = tab_ptr<T>(P, L.w_off[1]); p.w2 = tab_ptr<T>(P, L.w_off[2]);
    return p;
}

// Coefficients of a decomposition level, in place (before its restriction).
template <typename T, typename TW>
cudaError_t run_coef_level(const mgard_plan *P, int j, void *A, char *ws, cudaStream_t st)
{
    const PlaceParams p = place_params<T>(P, j, A, ws);
    return timed(P, KIND_PLACE, j, st, [&] { return launch_coef<T, TW>(P->act, p, P->num_sms, st); });
}

// Final coarse values V_j into the N_{l-1} nodes of the level array.
template <typename T, typename TW>
cudaError_t run_scatter_level(const mgard_plan *P, int j, void *A, char *ws, cudaStream_t st)
{
    const PlaceParams p = place_params<T>(P, j, A, ws);
    return timed(P, KIND_PLACE_EVEN, j, st, [&] { return launch_scatter<T, TW>(P->act, p, st); });
}

template <typename T, typename TW>
cudaError_t run_interp_level(const mgard_plan *P, int j, void *A, char *ws, cudaStream_t st)
{
    const PlaceParams p = place_params<T>(P, j, A, ws);
    return timed(P, KIND_INTERP, j, st, [&] { return launch_interp<T, TW>(P->act, p, P->num_sms, st); });
}

// Row-chunk kernel `kind` (0 sweeps, 1 restriction) for level j on level
// array A: an eligible level, not switched off, and a 16-byte aligned array
// (the workspace arrays always are; the user array at level 0 may not be).
bool rc_on(const mgard_plan *P, int j, const void *A, int kind)
{
    return P->lv[j].rc_q[0] > 0 && !(P->rc_off & (1 << kind)) && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
}

// The slab load-vector kernel for level j (configured: a 3D FP32 level array
// with rows of 128 k + 1 nodes, not switched off).
bool slab_on(const mgard_plan *P, int j) { return P->lv[j].slab_ty > 0; }

// Leading dims whose solve the level's load-vector kernel already did.
int solved_first(const mgard_plan *P, int j, const void *A)
{
    if (slab_on(P, j)) return P->lv[j].slab_xs ? 1 : 0;
    return (rc_on(P, j, A, 1) && P->lv[j].rc_xs) ? 1 : 0;
}

// Load vector and coarse gather of level j by the slab kernel.
template <typename TW>
cudaError_t run_slab(const mgard_plan *P, int j, int mode, const void *A, char *ws, cudaStream_t st)
{
    const mgard_level &L = P->lv[j];
    SlabParams p;
    p.A = A;
    p.F = ws + L.f_off;
    p.V = ws + L.v_off;
    p.n0 = (int)L.n[0]; p.n1 = (int)L.n[1]; p.n2 = (int)L.n[2];
    p.m0 = (int)L.m[0]; p.m1 = (int)L.m[1]; p.m2 = (int)L.m[2];
    p.k0 = tab_ptr<float>(P, L.k_off[0]); p.k1 = tab_ptr<float>(P, L.k_off[1]); p.k2 = tab_ptr<float>(P, L.k_off[2]);
    p.nb = L.slab_nb;
    p.zchunk = L.slab_zc;
    p.nzc = L.slab_nzc;
    p.nitems = L.slab_nb * L.slab_nzc;
    p.ns = L.slab_ns;
    p.slot_bytes = L.slab_sb;
    p.kuni1 = L.kuni32[1];
    p.hook = P->slab_hook;
    p.status = P->d_status;
    p.wait_ns = P->slab_wait_ns;
    p.fx = tab_ptr<TW>(P, L.t_off[2]);
    return timed(P, mode == MODE_DEC ? KIND_RESTRICT_DEC : KIND_RESTRICT_REC, j, st,
                 [&] { return launch_slab<TW>(L.slab_ty, L.slab_mb, L.slab_xs, p, L.slab_grid, st); });
}

template <typename T, typename TW>
RcParams rc_params(const mgard_plan *P, int j, void *A, char *ws, int kind)
{
    const mgard_level &L = P->lv[j];
    RcParams p;
    p.A = A;
    p.F = ws + L.f_off;
    p.V = ws + L.v_off;
    p.n0 = (int)L.n[0]; p.n1 = (int)L.n[1]; p.n2 = (int)L.n[2];
    p.m0 = (int)L.m[0]; p.m1 = (int)L.m[1]; p.m2 = (int)L.m[2];
    p.S = L.rc_s[kind];
    p.nb = kind == 0 ? (int)L.m[1] : (int)((L.m[1] + kRcRows - 1) / kRcRows);
    p.zchunk = L.rc_zc[kind];
    p.nzc = L.rc_nzc[kind];
    p.nitems = p.S * p.nb * p.nzc;
    p.w0 = tab_ptr<T>(P, L.w_off[0]); p.w1 = tab_ptr<T>(P, L.w_off[1]); p.w2 = tab_ptr<T>(P, L.w_off[2]);
    p.k0 = tab_ptr<T>(P, L.k_off[0]); p.k1 = tab_ptr<T>(P, L.k_off[1]); p.k2 = tab_ptr<T>(P, L.k_off[2]);
    p.fx = tab_ptr<TW>(P, L.t_off[2]);
    return p;
}

// Coefficients (MODE_DEC) or interpolation (MODE_REC) of level j.
template <typename T, typename TW>
cudaError_t run_rc_sweep(const mgard_plan *P, int j, int mode, void *A, char *ws, cudaStream_t st)
{
    const mgard_level &L = P->lv[j];
    const RcParams p = rc_params<T, TW>(P, j, A, ws, 0);
    return timed(P, mode == MODE_DEC ? KIND_PLACE : KIND_INTERP, j, st, [&] {
        return launch_rc<T, TW>(0, L.rc_q[0], mode, P->act == ACT_3D, L.wuni2 != 0, false, p, L.rc_grid[0], st);
    });
}

// Load vector and coarse gather of level j (with the dim-2 solve when rc_xs).
template <typename T, typename TW>
cudaError_t run_rc_restrict(const mgard_plan *P, int j, int mode, void *A, char *ws, cudaStream_t st)
{
    const mgard_level &L = P->lv[j];
    const RcParams p = rc_params<T, TW>(P, j, A, ws, 1);
    const bool ku = (sizeof(T) == 4 ? L.kuni32[2] : L.kuni64[2]) != 0;
    return timed(P, mode == MODE_DEC ? KIND_RESTRICT_DEC : KIND_RESTRICT_REC, j, st, [&] {
        return launch_rc<T, TW>(1, L.rc_q[1], mode, P->act == ACT_3D, ku, L.rc_xs, p, L.rc_grid[1], st);
    });
}

// Levels small_j .. L-1 in one block, on the array of level small_j (the
// user array when small_j = 0, else V_{small_j - 1}); `first` > small_j
// starts at a smaller array, which the shared memory sized for level
// small_j also holds.
template <typename T, typename TW>
cudaError_t run_small(const mgard_plan *P, int mode, void *A, cudaStream_t st, int adjoint = -1, int first = -1)
{
    const int j0 = (adjoint >= 0) ? P->adj_j : (first >= 0 ? first : P->small_j);
    const int64_t *n = (j0 == 0) ? P->n : P->lv[j0 - 1].m;
    SmallParams sp;
    sp.A = A;
    for (int d = 0; d < 3; ++d) sp.n[d] = (int)n[d];
    sp.nlev = P->L - j0;
    sp.hcap = P->small_hcap;
    for (int i = 0; i < sp.nlev; ++i) {
        const mgard_level &L = P->lv[j0 + i];
        for (int d = 0; d < 3; ++d) {
            sp.w[i][d] = tab_ptr<TW>(P, L.w_off[d]);
            sp.k[i][d] = tab_ptr<TW>(P, L.k_off[d]);
            sp.fac[i][d] = tab_ptr<TW>(P, L.t_off[d]);
        }
    }
    if (adjoint >= 0)  // transposed maps: adjoint 0 = decomposition, 1 = recomposition
        return timed(P, KIND_ADJ, j0, st, [&] { return launch_small_adj<T, TW>(adjoint, sp, P->adj_smem, st); });
    return timed(P, KIND_SMALL, j0, st, [&] { return launch_small<T, TW>(mode, sp, P->small_smem, st); });
}

// Levels coop_j .. L-1 in one cooperative launch (multi.cuh); level coop_j
// works on the user array (type TX) when coop_j = 0.
template <typename TX, typename TW>
cudaError_t run_multi(const mgard_plan *P, int mode, void *data, char *ws, cudaStream_t st)
{
    const int j0 = P->coop_j;
    MultiParams mp;
    mp.nd = P->coop_s - j0;
    for (int i = 0; i < mp.nd; ++i) {
        const int j = j0 + i;
        const mgard_level &L = P->lv[j];
        MultiLevel &ml = mp.lv[i];
        ml.X = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        ml.V = ws + L.v_off;
        ml.F = ws + L.f_off;
        ml.G = ws + P->coop_g_off[i];
        for (int d = 0; d < 3; ++d) {
            ml.n[d] = (int)L.n[d];
            ml.m[d] = (int)L.m[d];
            ml.w[d] = tab_ptr<TW>(P, L.w_off[d]);
            ml.k[d] = tab_ptr<TW>(P, L.k_off[d]);
            ml.fac[d] = tab_ptr<TW>(P, L.t_off[d]);
        }
    }
    mp.small = P->coop_s < P->L ? 1 : 0;
    if (mp.small) {
        const int s0 = P->coop_s;
        SmallParams &sp = mp.sp;
        sp.A = ws + P->lv[s0 - 1].v_off;
        for (int d = 0; d < 3; ++d) sp.n[d] = (int)P->lv[s0 - 1].m[d];
        sp.nlev = P->L - s0;
        sp.hcap = P->coop_hcap;
        for (int i = 0; i < sp.nlev; ++i) {
            const mgard_level &L = P->lv[s0 + i];
            for (int d = 0; d < 3; ++d) {
                sp.w[i][d] = tab_ptr<TW>(P, L.w_off[d]);
                sp.k[i][d] = tab_ptr<TW>(P, L.k_off[d]);
                sp.fac[i][d] = tab_ptr<TW>(P, L.t_off[d]);
            }
        }
    }
    mp.bar = reinterpret_cast<unsigned *>(ws + P->coop_bar_off);
    mp.spin_limit = P->coop_spin > 0 ? P->coop_spin : kMultiSpinLimit;
    cudaError_t err = cudaMemsetAsync(mp.bar, 0, kMultiBarrierWords * sizeof(unsigned), st);
    if (err != cudaSuccess) return err;
    return timed(P, KIND_MULTI, j0, st, [&] { return launch_multi<TX, TW>(mode, mp, P->coop_grid, P->coop_smem, st); });
}

// Decomposition, levels L..1 (Section II-A): level j = 0 works on the user
// array (element type TU), deeper levels on the compact coarse arrays V_{j-1}
// of the workspace (type TW).  Per level: the coefficients go in place (they
// depend only on the level's own values), the restriction reads them and
// gathers the coarse nodes into V_j, and the solves add the correction to
// V_j.  The coarse levels run in one cooperative launch (from coop_j) or one
// block (from small_j); then, coarsest first, every level array receives the
// final values of its coarse nodes.
template <typename TU, typename TW>
mgard_status exec_decompose(const mgard_plan *P, void *data, char *ws, cudaStream_t st, bool allow_coop)
{
    cudaError_t err;
    const bool coop = allow_coop && P->coop_j < P->L;
    const int J = coop ? P->coop_j : P->small_j;
    for (int j = 0; j < J; ++j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        if (rc_on(P, j, A, 0))
            err = (j == 0) ? run_rc_sweep<TU, TW>(P, j, MODE_DEC, A, ws, st)
                           : run_rc_sweep<TW, TW>(P, j, MODE_DEC, A, ws, st);
        else
            err = (j == 0) ? run_coef_level<TU, TW>(P, j, A, ws, st) : run_coef_level<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose: coefficient kernel");
        if (slab_on(P, j))
            err = run_slab<TW>(P, j, MODE_DEC, A, ws, st);
        else if (rc_on(P, j, A, 1))
            err = (j == 0) ? run_rc_restrict<TU, TW>(P, j, MODE_DEC, A, ws, st)
                           : run_rc_restrict<TW, TW>(P, j, MODE_DEC, A, ws, st);
        else
            err = (j == 0) ? run_restrict_level<TU, TW>(P, j, MODE_DEC, A, ws, st)
                           : run_restrict_level<TW, TW>(P, j, MODE_DEC, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose: load-vector kernel");
        err = run_solves<TW>(P, j, +1, ws, st, nullptr, solved_first(P, j, A));
        if (err != cudaSuccess) return cuda_fail(err, "decompose: correction solve kernel");
    }
    if (coop) {
        err = (J == 0) ? run_multi<TU, TW>(P, MODE_DEC, data, ws, st) : run_multi<TW, TW>(P, MODE_DEC, data, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose: cooperative coarse-level kernel");
    } else if (J < P->L) {
        void *A = (J == 0) ? data : (void *)(ws + P->lv[J - 1].v_off);
        err = (J == 0) ? run_small<TU, TW>(P, MODE_DEC, A, st) : run_small<TW, TW>(P, MODE_DEC, A, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose: single-block coarse-level kernel");
    }
    for (int j = J - 1; j >= 0; --j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = (j == 0) ? run_scatter_level<TU, TW>(P, j, A, ws, st) : run_scatter_level<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose: coarse placement kernel");
    }
    return MGARD_OK;
}

// Recomposition, levels 1..L: first every level's load vector F_j and the
// gathered coarse array V_j (both depend only on stored coefficients), then
// coarsest first: correction solve with V_j -= z, then interpolation.  With
// D > 0 only steps D .. L-1 run, on the level array V_{D-1} (already
// gathered), which ends up holding the recomposed level-(L-D) values.
template <typename TU, typename TW>
mgard_status exec_recompose(const mgard_plan *P, void *data, char *ws, cudaStream_t st, bool allow_coop, int D = 0)
{
    cudaError_t err;
    const bool coop = allow_coop && P->coop_j < P->L && D <= P->coop_j;
    const int J = coop ? P->coop_j : std::max(P->small_j, D);
    for (int j = D; j < J; ++j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        if (slab_on(P, j))
            err = run_slab<TW>(P, j, MODE_REC, A, ws, st);
        else if (rc_on(P, j, A, 1))
            err = (j == 0) ? run_rc_restrict<TU, TW>(P, j, MODE_REC, A, ws, st)
                           : run_rc_restrict<TW, TW>(P, j, MODE_REC, A, ws, st);
        else
            err = (j == 0) ? run_restrict_level<TU, TW>(P, j, MODE_REC, A, ws, st)
                           : run_restrict_level<TW, TW>(P, j, MODE_REC, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose: load-vector kernel");
    }
    if (coop) {
        err = (J == 0) ? run_multi<TU, TW>(P, MODE_REC, data, ws, st) : run_multi<TW, TW>(P, MODE_REC, data, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose: cooperative coarse-level kernel");
    } else if (J < P->L) {
        void *A = (J == 0) ? data : (void *)(ws + P->lv[J - 1].v_off);
        err = (J == 0) ? run_small<TU, TW>(P, MODE_REC, A, st, -1, J) : run_small<TW, TW>(P, MODE_REC, A, st, -1, J);
        if (err != cudaSuccess) return cuda_fail(err, "recompose: single-block coarse-level kernel");
    }
    for (int j = J - 1; j >= D; --j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = run_solves<TW>(P, j, -1, ws, st, nullptr, solved_first(P, j, A));
        if (err != cudaSuccess) return cuda_fail(err, "recompose: correction solve kernel");
        if (rc_on(P, j, A, 0))
            err = (j == 0) ? run_rc_sweep<TU, TW>(P, j, MODE_REC, A, ws, st)
                           : run_rc_sweep<TW, TW>(P, j, MODE_REC, A, ws, st);
        else
            err = (j == 0) ? run_interp_level<TU, TW>(P, j, A, ws, st) : run_interp_level<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose: interpolation kernel");
    }
    return MGARD_OK;
}

template <typename TU, typename TW>
cudaError_t run_prolong(const mgard_plan *P, int D, void *data, char *ws, cudaStream_t st)
{
    const int64_t *m = P->lv[D - 1].m;
    ProlongParams p;
    p.out = data;
    p.V = ws + P->lv[D - 1].v_off;
    p.w0 = tab_ptr<TW>(P, P->pro_off[D - 1][0]);
    p.w1 = tab_ptr<TW>(P, P->pro_off[D - 1][1]);
    p.w2 = tab_ptr<TW>(P, P->pro_off[D - 1][2]);
    p.n0 = (int)P->n[0]; p.n1 = (int)P->n[1]; p.n2 = (int)P->n[2];
    p.m0 = (int)m[0]; p.m1 = (int)m[1]; p.m2 = (int)m[2];
    p.shift = D;
    p.seg = 0;
    return timed(P, KIND_PROLONG, 0, st, [&] { return launch_prolong<TU, TW>(p, P->num_sms, st); });
}

template <typename T, typename TW>
cudaError_t run_gather(const mgard_plan *P, int j, void *A, char *ws, cudaStream_t st);

// Recomposition from the first L + 1 - D coefficient classes (Section I,
// Fig. 1; Section II-A, overall process): the classes of the D finest levels
// are left out, i.e. their coefficients are zero.  The coarse nodes are
// gathered down to N_{L-D} (the dropped coefficients are never read), levels
// 1 .. L-D recompose as usual into V_{D-1}, and with zero coefficients the
// remaining D steps are pure interpolation, done in one pass onto the
// finest array.
template <typename TU, typename TW>
mgard_status exec_recompose_classes(const mgard_plan *P, void *data, char *ws, cudaStream_t st, int D)
{
    if (D == 0) return exec_recompose<TU, TW>(P, data, ws, st, true);
    cudaError_t err;
    for (int j = 0; j < D; ++j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = (j == 0) ? run_gather<TU, TW>(P, j, A, ws, st) : run_gather<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_classes: gather kernel");
    }
    const mgard_status s = exec_recompose<TU, TW>(P, data, ws, st, true, D);
    if (s != MGARD_OK) return s;
    err = run_prolong<TU, TW>(P, D, data, ws, st);
    if (err != cudaSuccess) return cuda_fail(err, "recompose_classes: interpolation kernel");
    return MGARD_OK;
}

template <typename T, typename TW>
AdjParams adj_params(const mgard_plan *P, int j, void *A, const void *Z, int sign)
{
    const mgard_level &L = P->lv[j];
    AdjParams p;
    p.A = A;
    p.Z = Z;
    p.n0 = L.n[0]; p.n1 = L.n[1]; p.n2 = L.n[2];
    p.m0 = L.m[0]; p.m1 = L.m[1]; p.m2 = L.m[2];
    p.k0 = tab_ptr<TW>(P, L.k_off[0]); p.k1 = tab_ptr<TW>(P, L.k_off[1]); p.k2 = tab_ptr<TW>(P, L.k_off[2]);
    p.w0 = tab_ptr<T>(P, L.w_off[0]); p.w1 = tab_ptr<T>(P, L.w_off[1]); p.w2 = tab_ptr<T>(P, L.w_off[2]);
    p.sign = sign;
    return p;
}

template <typename T, typename TW>
cudaError_t run_gather(const mgard_plan *P, int j, void *A, char *ws, cudaStream_t st)
{
    const PlaceParams p = place_params<T>(P, j, A, ws);
    return timed(P, KIND_ADJ, j, st, [&] { return launch_gather<T, TW>(P->act, p, st); });
}

template <typename T, typename TW>
cudaError_t run_adj_odd(const mgard_plan *P, int j, void *A, const void *Z, int sign, cudaStream_t st)
{
    const AdjParams p = adj_params<T, TW>(P, j, A, Z, sign);
    return timed(P, KIND_ADJ, j, st, [&] { return launch_adj_odd<T, TW>(P->act, p, st); });
}

template <typename T, typename TW>
cudaError_t run_adj_even(const mgard_plan *P, int j, void *A, const void *B, int sign, cudaStream_t st)
{
    const AdjParams p = adj_params<T, TW>(P, j, A, B, sign);
    return timed(P, KIND_ADJ, j, st, [&] { return launch_adj_even<T, TW>(P->act, p, st); });
}

// Transpose of the decomposition (back-propagation through it), coarsest
// level first: gather the coarse nodes of every level, then per level
// z = M_{l-1}^{-1} V_j, odd <- odd + K^T z, even <- V_j - Pi^T odd.
template <typename TU, typename TW>
mgard_status exec_decompose_adjoint(const mgard_plan *P, void *data, char *ws, cudaStream_t st)
{
    cudaError_t err;
    // levels from adj_j on: one block, coarsest first, on the array of
    // level adj_j (its gathers are identities there)
    const int J = P->adj_j;
    for (int j = 0; j < J; ++j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = (j == 0) ? run_gather<TU, TW>(P, j, A, ws, st) : run_gather<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose_adjoint: gather kernel");
    }
    if (J < P->L) {
        void *A = (J == 0) ? data : (void *)(ws + P->lv[J - 1].v_off);
        err = (J == 0) ? run_small<TU, TW>(P, MODE_DEC, A, st, 0) : run_small<TW, TW>(P, MODE_DEC, A, st, 0);
        if (err != cudaSuccess) return cuda_fail(err, "decompose_adjoint: single-block kernel");
    }
    for (int j = J - 1; j >= 0; --j) {
        const mgard_level &L = P->lv[j];
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = run_solves<TW>(P, j, 0, ws, st, ws + L.v_off);
        if (err != cudaSuccess) return cuda_fail(err, "decompose_adjoint: solve kernel");
        err = (j == 0) ? run_adj_odd<TU, TW>(P, j, A, ws + L.f_off, +1, st)
                       : run_adj_odd<TW, TW>(P, j, A, ws + L.f_off, +1, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose_adjoint: odd-node kernel");
        err = (j == 0) ? run_adj_even<TU, TW>(P, j, A, ws + L.v_off, -1, st)
                       : run_adj_even<TW, TW>(P, j, A, ws + L.v_off, -1, st);
        if (err != cudaSuccess) return cuda_fail(err, "decompose_adjoint: even-node kernel");
    }
    return MGARD_OK;
}

// Transpose of the recomposition, finest level first: even <- even + Pi^T
// odd, gather it into V_j, z = M_{l-1}^{-1} V_j, odd <- odd - K^T z; after
// the coarser levels, V_j goes back to the even nodes.
template <typename TU, typename TW>
mgard_status exec_recompose_adjoint(const mgard_plan *P, void *data, char *ws, cudaStream_t st)
{
    cudaError_t err;
    const int J = P->adj_j;  // levels from adj_j on: one block, finest first
    for (int j = 0; j < J; ++j) {
        const mgard_level &L = P->lv[j];
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        err = (j == 0) ? run_adj_even<TU, TW>(P, j, A, nullptr, +1, st)
                       : run_adj_even<TW, TW>(P, j, A, nullptr, +1, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: even-node kernel");
        err = (j == 0) ? run_gather<TU, TW>(P, j, A, ws, st) : run_gather<TW, TW>(P, j, A, ws, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: gather kernel");
        err = run_solves<TW>(P, j, 0, ws, st, ws + L.v_off);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: solve kernel");
        err = (j == 0) ? run_adj_odd<TU, TW>(P, j, A, ws + L.f_off, -1, st)
                       : run_adj_odd<TW, TW>(P, j, A, ws + L.f_off, -1, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: odd-node kernel");
    }
    if (J < P->L) {
        void *A = (J == 0) ? data : (void *)(ws + P->lv[J - 1].v_off);
        err = (J == 0) ? run_small<TU, TW>(P, MODE_REC, A, st, 1) : run_small<TW, TW>(P, MODE_REC, A, st, 1);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: single-block kernel");
    }
    for (int j = J - 1; j >= 0; --j) {
        void *A = (j == 0) ? data : (void *)(ws + P->lv[j - 1].v_off);
        const PlaceParams p = (j == 0) ? place_params<TU>(P, j, A, ws) : place_params<TW>(P, j, A, ws);
        err = (j == 0) ? launch_scatter<TU, TW>(P->act, p, st) : launch_scatter<TW, TW>(P->act, p, st);
        if (err != cudaSuccess) return cuda_fail(err, "recompose_adjoint: scatter kernel");
    }
    return MGARD_OK;
}

// Launch configuration of a level's load-vector kernel for tile
// configuration L.rcfg (tile grid, plane chunks, grid size).
template <typename TU, typename TW>
cudaError_t configure_restrict(const mgard_plan *P, mgard_level &L, bool finest, int64_t *items_out,
                               int64_t *slots_out)
{
    RestrictShape sh;
    cudaError_t err = finest ? restrict_shape<TU, TW>(P->act, MODE_DEC, L.rcfg, &sh)
                             : restrict_shape<TW, TW>(P->act, MODE_DEC, L.rcfg, &sh);
    if (err != cudaSuccess) return err;
    if (L.rcfg == 3) {
        // strips of tx x ty coarse nodes, the last one shifted back to end at
        // the final node: ceil(m/t) of them; the level must hold one strip
        if (L.m[2] < sh.tx || L.m[1] < sh.ty) return cudaErrorInvalidValue;
        L.tiles_y = (int)((L.m[1] + sh.ty - 1) / sh.ty);
        L.tiles_x = (int)((L.m[2] + sh.tx - 1) / sh.tx);
    } else {
        // tiles of ty x tx coarse nodes; the last tile of a dimension also
        // takes the final node, so there are ceil((m-1)/t) tiles
        L.tiles_y = (P->act == ACT_1D) ? 1 : (int)std::max<int64_t>(1, (L.m[1] - 1 + sh.ty - 1) / sh.ty);
        L.tiles_x = (int)std::max<int64_t>(1, (L.m[2] - 1 + sh.tx - 1) / sh.tx);
    }
    const int64_t tiles = (int64_t)L.tiles_y * L.tiles_x;
    const int64_t ipb = std::max(1, sh.items_per_block);
    const int64_t slots = (int64_t)std::max(1, sh.blocks_per_sm) * P->num_sms * ipb;  // resident items
    if (P->act == ACT_3D) {
        // enough items for about two per resident slot, chunks of >= 2 coarse
        // planes (each chunk also reads 3 fine planes of its neighbours); the
        // last chunk takes the final plane
        int64_t nzc = std::max<int64_t>(1, (2 * slots + tiles - 1) / tiles);
        nzc = std::min<int64_t>(nzc, std::max<int64_t>(1, (L.m[0] - 1) / 2));
        L.zchunk = (int)std::max<int64_t>(1, (L.m[0] - 1 + nzc - 1) / nzc);
        if (L.zreq > 0) L.zchunk = L.zreq;
        L.nzc = (int)std::max<int64_t>(1, (L.m[0] - 1 + L.zchunk - 1) / L.zchunk);
    } else {
        L.zchunk = 1;
        L.nzc = 1;
    }
    if (P->act == ACT_1D) {
        // per-coarse-node kernel: blocks of sh.tx coarse nodes
        L.tiles_x = (int)std::max<int64_t>(1, (L.m[2] + sh.tx - 1) / sh.tx);
    }
    const int64_t items = (P->act == ACT_1D) ? L.tiles_x : tiles * L.nzc;
    const int64_t blocks = (items + ipb - 1) / ipb;
    L.rgrid_dec = L.rgrid_rec = (int)std::min<int64_t>(blocks, std::max(1, sh.blocks_per_sm) * (int64_t)P->num_sms);
    *items_out = items;
    *slots_out = slots;
    return cudaSuccess;
}

// Unless the tile configuration was set by mgard_plan_tune, take the tallest
// tile (fewest halo rows re-read) that still gives every resident slot of the
// GPU a work item (small levels need short tiles to spread over the SMs),
// else the one with the most items.
template <typename TU, typename TW>
cudaError_t configure_level(mgard_plan *P, mgard_level &L, bool finest)
{
    int64_t items = 0, slots = 0;
    if (L.rcfg_user || P->act == ACT_1D) return configure_restrict<TU, TW>(P, L, finest, &items, &slots);
    int best = 0;
    int64_t best_items = -1;
    // warp strips first for 4-byte level arrays (FP64 arithmetic is slow
    // enough on this GPU that the strips' recomputed halo rows cost more than
    // the tiles' staging); then tiles of 16, 8, 4 coarse rows
    static const int order4[kRestrictConfigs] = {3, 2, 0, 1};
    static const int order8[kRestrictConfigs] = {2, 0, 1, 3};
    const bool elem4 = (finest ? P->elem_user : P->elem_ws) == 4;
    for (int cfg : (elem4 ? order4 : order8)) {
        L.rcfg = cfg;
        cudaError_t err = configure_restrict<TU, TW>(P, L, finest, &items, &slots);
        if (err != cudaSuccess) {  // e.g. more shared memory than the device has
            cudaGetLastError();
            continue;
        }
        if (items >= slots) {
            best = cfg;
            break;
        }
        if (items > best_items) {
            best_items = items;
            best = cfg;
        }
    }
    L.rcfg = best;
    return configure_restrict<TU, TW>(P, L, finest, &items, &slots);
}

// Row-chunk configuration of a 2D/3D level (rowchunk.cuh): rows of
// 2^k 256 + 1 nodes with n1 = 1 mod 8 (then n1, n2, m1, m2 = 1 mod 4, which
// the kernels' word offsets rely on).  Segments of 256 columns for the
// sweeps; for the restriction segments of 512 columns where the rows split
// into them and hold 4-byte elements (a row of one segment also solves
// along dim 2), else 256.  Plane chunks and grids per kernel.  Leaves
// rc_q[0] = 0 (the other kernels) otherwise.
template <typename TU, typename TW>
cudaError_t configure_rc(mgard_plan *P, mgard_level &L, bool finest)
{
    L.rc_q[0] = L.rc_q[1] = 0;
    if (P->act == ACT_1D) return cudaSuccess;
    const int es = (int)(finest ? P->elem_user : P->elem_ws);
    const int64_t n1 = L.n[1], n2 = L.n[2];
    if ((n2 - 1) % 256 != 0 || n1 < 9 || (n1 - 1) % 8 != 0) return cudaSuccess;
    const int E = 16 / es;
    const int qs = 256 / (32 * E);                                   // 256-column segments
    const int wr = (es == 4 && (n2 - 1) % 512 == 0) ? 512 : 256;
    const int qr = wr / (32 * E);
    const int Ss = (int)((n2 - 1) / 256), Sr = (int)((n2 - 1) / wr);
    const bool hz = P->act == ACT_3D, xs = (Sr == 1), wu = L.wuni2 != 0;
    const bool ku = (es == 4 ? L.kuni32[2] : L.kuni64[2]) != 0;
    int bd = 0, br = 0, bx = 0;
    cudaError_t err;
    if (finest) {
        err = rc_occupancy<TU, TW>(0, qs, MODE_DEC, hz, wu, false, Ss, &bd);
        if (err == cudaSuccess) err = rc_occupancy<TU, TW>(0, qs, MODE_REC, hz, wu, false, Ss, &br);
        if (err == cudaSuccess) err = rc_occupancy<TU, TW>(1, qr, MODE_DEC, hz, ku, xs, Sr, &bx);
    } else {
        err = rc_occupancy<TW, TW>(0, qs, MODE_DEC, hz, wu, false, Ss, &bd);
        if (err == cudaSuccess) err = rc_occupancy<TW, TW>(0, qs, MODE_REC, hz, wu, false, Ss, &br);
        if (err == cudaSuccess) err = rc_occupancy<TW, TW>(1, qr, MODE_DEC, hz, ku, xs, Sr, &bx);
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;  // not available here: the other kernels
    }
    const int bs = std::min(bd, br);
    if (bs < 1 || bx < 1) return cudaSuccess;
    const int64_t m0 = L.m[0], m1 = L.m[1];
    // sweep: work items of one coarse row of a segment and a chunk of coarse
    // intervals, about four per resident warp
    const int64_t slots_s = (int64_t)bs * P->num_sms * kRcWarps;
    int64_t nzc = 1, zc = 0;
    if (hz) {
        nzc = std::max<int64_t>(1, std::min<int64_t>((4 * slots_s + Ss * m1 - 1) / (Ss * m1), m0 - 1));
        zc = (m0 - 1 + nzc - 1) / nzc;
        if (P->rc_zreq > 0) zc = std::min<int64_t>(P->rc_zreq, m0 - 1);
        nzc = (m0 - 1 + zc - 1) / zc;
    }
    L.rc_zc[0] = (int)zc;
    L.rc_nzc[0] = (int)nzc;
    const int64_t items_s = (int64_t)Ss * m1 * nzc;
    L.rc_grid[0] = (int)std::min<int64_t>((items_s + kRcWarps - 1) / kRcWarps, (int64_t)bs * P->num_sms);
    // restriction: blocks of kRcRows coarse rows of a segment and a chunk of
    // coarse planes (each chunk re-reads 3 fine planes), about two per warp
    const int64_t nb = (m1 + kRcRows - 1) / kRcRows;
    const int64_t slots_r = (int64_t)bx * P->num_sms * kRcWarps;
    int64_t nzr = 1, zr = 1;
    if (hz) {
        nzr = std::max<int64_t>(1, std::min<int64_t>((2 * slots_r + Sr * nb - 1) / (Sr * nb), std::max<int64_t>(1, (m0 - 1) / 2)));
        zr = std::max<int64_t>(1, (m0 - 1 + nzr - 1) / nzr);
        if (P->rc_zreq > 0) zr = std::min<int64_t>(P->rc_zreq, std::max<int64_t>(1, m0 - 1));
        nzr = std::max<int64_t>(1, (m0 - 1 + zr - 1) / zr);
    }
    L.rc_zc[1] = (int)zr;
    L.rc_nzc[1] = (int)nzr;
    const int64_t items_r = (int64_t)Sr * nb * nzr;
    L.rc_grid[1] = (int)std::min<int64_t>((items_r + kRcWarps - 1) / kRcWarps, (int64_t)bx * P->num_sms);
    if (items_s >= (int64_t(1) << 31) || items_r >= (int64_t(1) << 31)) return cudaSuccess;
    L.rc_q[0] = qs;
    L.rc_q[1] = qr;
    L.rc_s[0] = Ss;
    L.rc_s[1] = Sr;
    L.rc_xs = xs;
    return cudaSuccess;
}

// Slab load-vector configuration of a 3D level whose array holds 4-byte
// elements and whose rows have n2 = 64 k + 1 nodes (k <= 16): coarse rows per
// band, ring slots and register variant (bands of 6 rows, 2 slots and three
// blocks per SM where they fit, or as tuned), and the coarse planes per chunk.
// Leaves slab_ty = 0 (the other kernels) otherwise.
template <typename TW>
cudaError_t configure_slab(mgard_plan *P, mgard_level &L, bool finest)
{
    L.slab_ty = 0;
    const int es = (int)(finest ? P->elem_user : P->elem_ws);
    if (P->slab_off || P->per_dim || P->act != ACT_3D || es != 4) return cudaSuccess;
    const int64_t n2 = L.n[2], m0 = L.m[0], m1 = L.m[1];
    if ((n2 - 1) % 64 != 0 || (n2 - 1) / 2 > kSlabMaxThreads || m0 < 2) return cudaSuccess;
    // (rows per band, ring slots, blocks per SM) in order of preference, as
    // tuned: the first whose shared memory fits a block; the dim-2 solve in
    // the kernel when switched on
    const bool xs = P->slab_xs_on;
    int ty = 0, ns = 0, bps = 0, minb = 0;
    static const int pref[7][3] = {{6, 2, 3}, {8, 2, 2}, {4, 2, 3}, {4, 3, 3}, {8, 3, 2}, {8, 4, 2}, {4, 4, 2}};
    for (const auto &c : pref) {
        const int cty = P->slab_tyreq > 0 ? P->slab_tyreq : c[0];
        const int cns = P->slab_nsreq > 0 ? P->slab_nsreq : c[1];
        // FP64 coarse rows (mixed scheme): the two-block register budget
        const int cmb = P->slab_mbreq > 0 ? P->slab_mbreq : (sizeof(TW) == 8 ? 2 : c[2]);
        if (m1 < cty) continue;
        int b = 0;
        if (slab_occupancy<TW>(cty, (int)n2, cns, cmb, xs, &b) != cudaSuccess || b < 1) {
            cudaGetLastError();
            continue;
        }
        ty = cty;
        ns = cns;
        minb = cmb;
        bps = b;
        break;
    }
    if (ty == 0) return cudaSuccess;  // not available here: the other kernels
    const int64_t nb = (m1 + ty - 1) / ty;
    const int64_t slots = (int64_t)bps * P->num_sms;
    // about two items per resident block (blocks that finish early leave the
    // memory system to the others, so enough items matter more than even
    // shares; each chunk also streams 3 of its neighbours' planes), at least
    // 2 coarse planes per chunk
    const int64_t zmax = std::max<int64_t>(1, m0 - 1);
    int64_t best_zc = 0;
    if (L.slab_zreq > 0) {
        best_zc = std::min<int64_t>(L.slab_zreq, zmax);
    } else {
        const int64_t want = std::max<int64_t>(1, (2 * slots + nb - 1) / nb);  // chunks
        best_zc = std::max<int64_t>(std::min<int64_t>(2, zmax), (zmax + want - 1) / want);
    }
    if (best_zc <= 0) return cudaSuccess;
    const int64_t nzc = std::max<int64_t>(1, (m0 - 1 + best_zc - 1) / best_zc);
    const int64_t items = nb * nzc;
    if (items >= (int64_t(1) << 31)) return cudaSuccess;
    L.slab_ty = ty;
    L.slab_ns = ns;
    L.slab_mb = minb;
    L.slab_xs = xs;
    L.slab_sb = slab_slot_bytes_of(ty, (int)n2);
    L.slab_nb = (int)nb;
    L.slab_zc = (int)best_zc;
    L.slab_nzc = (int)nzc;
    L.slab_grid = (int)std::min(items, slots);
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *mgard_status_string(mgard_status s)
{
    switch (s) {
    case MGARD_OK: return "MGARD_OK";
    case MGARD_ERR_INVALID_ARG: return "MGARD_ERR_INVALID_ARG";
    case MGARD_ERR_UNSUPPORTED_SHAPE: return "MGARD_ERR_UNSUPPORTED_SHAPE";
    case MGARD_ERR_WORKSPACE: return "MGARD_ERR_WORKSPACE";
    case MGARD_ERR_CUDA: return "MGARD_ERR_CUDA";
    case MGARD_ERR_TIMEOUT: return "MGARD_ERR_TIMEOUT";
    case MGARD_ERR_INTERNAL: return "MGARD_ERR_INTERNAL";
    }
    return "MGARD_ERR_UNKNOWN";
}

const char *mgard_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Host part of plan creation: validation, level geometry, the tables (in
// double, returned in *tab) and the workspace layout.  Allocates no device
// memory; the table pointers of the plan are left null.
static mgard_status build_plan_host(int ndim, const int64_t *dims, int nlevels, const double *const *coords,
                                    mgard_dtype dtype, mgard_plan **out, std::vector<double> *tab_out,
                                    const int *dim_levels = nullptr)
{
    if (!out) return fail(MGARD_ERR_INVALID_ARG, "plan_create: out is NULL");
    *out = nullptr;
    if (!dims) return fail(MGARD_ERR_INVALID_ARG, "plan_create: dims is NULL");
    if (ndim < 1 || ndim > 3) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create: ndim must be 1..3");
    if (dtype != MGARD_F32 && dtype != MGARD_F64 && dtype != MGARD_F32_MIXED)
        return fail(MGARD_ERR_INVALID_ARG, "plan_create: unknown dtype");
    if (nlevels < -1) return fail(MGARD_ERR_INVALID_ARG, "plan_create: nlevels must be >= -1");

    // squeeze size-1 dimensions
    std::vector<int64_t> n;
    std::vector<std::vector<double>> x;
    std::vector<int> lk_req;  // requested level count of each kept dim (-1: its maximum)
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create: dims must be >= 1");
        if (dims[k] > (int64_t(1) << 31)) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create: dimension too large");
        if (dims[k] == 1) continue;
        lk_req.push_back(dim_levels ? dim_levels[k] : -2);
        std::vector<double> xk(dims[k]);
        if (coords && coords[k]) {
            for (int64_t i = 0; i < dims[k]; ++i) xk[i] = coords[k][i];
            for (int64_t i = 1; i < dims[k]; ++i)
                if (!(xk[i] > xk[i - 1]) || !std::isfinite(xk[i]))
                    return fail(MGARD_ERR_INVALID_ARG, "plan_create: coordinates must be finite and strictly increasing");
        } else if (coords) {
            return fail(MGARD_ERR_INVALID_ARG, "plan_create: coords given but coords[k] is NULL");
        } else {
            for (int64_t i = 0; i < dims[k]; ++i) xk[i] = (double)i / (double)(dims[k] - 1);
        }
        n.push_back(dims[k]);
        x.push_back(std::move(xk));
    }
    if (n.empty()) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create: no dimension larger than 1");
    const int nd = (int)n.size();

    int Lmax = 0;
    for (;;) {
        bool ok = true;
        for (int64_t v : n) {
            const int64_t step = int64_t(1) << (Lmax + 1);
            if ((v - 1) % step != 0 || (v - 1) < step) ok = false;
        }
        if (!ok || Lmax >= 30) break;
        ++Lmax;
    }
    int L = (nlevels < 0) ? Lmax : nlevels;
    // per-dimension level counts: dim k coarsens in the first Lk[k] steps
    std::vector<int> Lk(nd, 0);
    bool per_dim = false;
    if (dim_levels) {
        L = 0;
        for (int k = 0; k < nd; ++k) {
            int own = 0;
            while (own < 30 && (n[k] - 1) % (int64_t(1) << (own + 1)) == 0 && (n[k] - 1) >= (int64_t(1) << (own + 1)))
                ++own;
            const int want = lk_req[k] < 0 ? own : lk_req[k];
            if (lk_req[k] < -1 || want > own)
                return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create_per_dim: dim " + std::to_string(k) + " allows " +
                                                             std::to_string(own) + " levels");
            Lk[k] = want;
            L = std::max(L, want);
        }
        for (int k = 0; k < nd; ++k) per_dim = per_dim || Lk[k] != L;
    } else {
        for (int k = 0; k < nd; ++k) Lk[k] = L;
    }
    if (L > Lmax && !per_dim)
        return fail(MGARD_ERR_UNSUPPORTED_SHAPE,
                    "plan_create: every (dims[k]-1) must be divisible by 2^nlevels (max levels here: " +
                        std::to_string(Lmax) + ")");

    mgard_plan *P = new (std::nothrow) mgard_plan();
    if (!P) return fail(MGARD_ERR_INTERNAL, "plan_create: out of host memory");
    P->ndim = nd;
    P->act = act_of(nd);
    P->n[0] = P->n[1] = 1;
    for (int k = 0; k < nd; ++k) P->n[3 - nd + k] = n[k];
    if (nd < 3) P->n[0] = 1;
    if (nd < 2) P->n[1] = 1;
    P->L = L;
    P->per_dim = per_dim;
    P->dtype = dtype;
    P->elem_user = (dtype == MGARD_F64) ? 8 : 4;
    P->elem_ws = (dtype == MGARD_F32) ? 4 : 8;
    cudaError_t err = cudaGetDevice(&P->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (err != cudaSuccess) {
        delete P;
        return cuda_fail(err, "plan_create: device query");
    }
    P->row_grid = P->num_sms * 8;

    // per-level geometry and tables
    std::vector<double> tab;
    tab.reserve(1024);
    tab.push_back(0.0);  // offset 0 is a harmless dummy for inactive dims
    for (int k = 0; k < 8; ++k) tab.push_back(0.0);
    size_t ws = 0;
    P->lv.resize(L);
    for (int j = 0; j < L; ++j) {
        mgard_level &lv = P->lv[j];
        for (int q = 0; q < 3; ++q) {
            lv.n[q] = 1;
            lv.m[q] = 1;
            lv.co[q] = 0;
            lv.w_off[q] = lv.k_off[q] = lv.t_off[q] = 0;
            lv.kuni32[q] = lv.kuni64[q] = 0;
        }
        lv.wuni2 = 0;
        for (int k = 0; k < nd; ++k) {
            const int q = 3 - nd + k;
            const int64_t stride = int64_t(1) << std::min(j, Lk[k]);
            const int64_t nf = (n[k] - 1) / stride + 1;
            lv.n[q] = nf;
            if (j >= Lk[k]) {  // kept with all its nodes: P = I, no tables
                lv.m[q] = nf;
                continue;
            }
            std::vector<double> xf(nf);
            for (int64_t i = 0; i < nf; ++i) xf[i] = x[k][i * stride];
            lv.m[q] = (nf - 1) / 2 + 1;
            lv.co[q] = 1;
            build_dim_tables(xf, tab, &lv.w_off[q], &lv.k_off[q], &lv.t_off[q]);
            if (q == 2) {
                lv.wuni2 = 1;
                for (int64_t i = 1; i + 1 < nf; i += 2)
                    if (tab[lv.w_off[q] + 2 * i] != 0.5 || tab[lv.w_off[q] + 2 * i + 1] != 0.5) lv.wuni2 = 0;
            }
            // interior K rows all equal (bitwise, in each table precision)
            lv.kuni32[q] = lv.kuni64[q] = 1;
            for (int64_t I = 2; I + 1 < lv.m[q]; ++I)
                for (int t = 0; t < 5; ++t) {
                    const double a = tab[lv.k_off[q] + 5 * I + t], b = tab[lv.k_off[q] + 5 + t];
                    if (a != b) lv.kuni64[q] = 0;
                    if ((float)a != (float)b) lv.kuni32[q] = 0;
                }
        }
        const size_t mbytes = (size_t)count(lv.m) * P->elem_ws;
        lv.v_off = ws;
        ws = align_up(ws + mbytes);
        lv.f_off = ws;
        ws = align_up(ws + mbytes);
        lv.rcfg = 0;
        lv.rcfg_user = false;
        lv.svar = 0;
        lv.zreq = 0;
        for (int k = 0; k < nd; ++k) {
            const int q = 3 - nd + k;
            if (lv.m[q] > kMaxLine) {
                delete P;
                return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create: a coarse line is longer than 4096 nodes");
            }
        }
    }
    P->ws_bytes = ws;

    // weight of the right N_{L-D} neighbour of every finest node (0 on
    // N_{L-D} itself), D = 1..L, from the coordinates
    P->pro_off.assign(L, std::array<int64_t, 3>{0, 0, 0});
    for (int D = 1; D <= (per_dim ? 0 : L); ++D) {
        const int64_t s = int64_t(1) << D;
        for (int k = 0; k < nd; ++k) {
            P->pro_off[D - 1][3 - nd + k] = (int64_t)tab.size();
            for (int64_t i = 0; i < n[k]; ++i) {
                const int64_t a = i / s * s;
                tab.push_back(i == a ? 0.0 : (x[k][i] - x[k][a]) / (x[k][a + s] - x[k][a]));
            }
        }
    }

    // the finest level whose array the single-block kernel takes
    P->small_auto = L;
    for (int j = 0; j < (per_dim ? 0 : L); ++j) {
        const int64_t *nj = (j == 0) ? P->n : P->lv[j - 1].m;
        const int64_t es = (int64_t)P->elem_ws;
        const int64_t base = small_elems(nj) + small_tab_elems(nj, L - j), hp = small_hplane(nj);
        const bool sides_ok = nj[0] <= kSmallMaxSide && nj[1] <= kSmallMaxSide && nj[2] <= kSmallMaxSide;
        if (sides_ok && (base + hp) * es <= kSmallMaxBytes && L - j <= kSmallMaxLevels) {
            // H: as many first-level fine planes as fit, at most all of them
            const int64_t planes = std::min<int64_t>(nj[0], (kSmallMaxBytes / es - base) / hp);
            P->small_auto = j;
            P->small_hcap = (int)(planes * hp);
            P->small_smem = (size_t)((base + planes * hp) * es);
            break;
        }
    }
    P->small_j = P->small_auto;
    adj_select(P);

    // the cooperative kernel: from the first level whose coarse lines fit one
    // thread's registers, the grid runs every level until the array is small
    // enough for block 0 to finish in shared memory (H: all fine planes)
    P->coop_auto = L;
    for (int j = 0; j < (per_dim ? 0 : L); ++j) {
        const int64_t *nj = (j == 0) ? P->n : P->lv[j - 1].m;
        if (nj[0] <= kMultiMaxSide && nj[1] <= kMultiMaxSide && nj[2] <= kMultiMaxSide) {
            P->coop_auto = j;
            break;
        }
    }
    if (P->coop_auto < L) {
        const int j0 = P->coop_auto;
        const int64_t es = (int64_t)P->elem_ws;
        int s = j0;
        int64_t sbytes = 0;
        for (; s < L; ++s) {
            const int64_t *ns = (s == 0) ? P->n : P->lv[s - 1].m;
            sbytes = (small_elems(ns) + ns[0] * small_hplane(ns) + small_tab_elems(ns, L - s)) * es;
            if (count(ns) <= kMultiSmallNodes && sbytes <= kMultiSmallBytes) break;
        }
        // shared memory of a block: the largest grid level's planes, or the
        // levels block 0 finishes
        int64_t smem = (s < L) ? sbytes : 0;
        for (int j = j0; j < s; ++j)
            smem = std::max(smem, (kMultiTabElems + multi_level_elems(P->lv[j].n, P->lv[j].m)) * es);
        if (P->ndim >= 2 && s > j0 && s - j0 <= kMultiMaxLevels && L - s <= kSmallMaxLevels &&
            smem <= kSmallMaxBytes) {
            P->coop_s = s;
            P->coop_smem = (size_t)smem;
            if (s < L) {
                const int64_t *ns = P->lv[s - 1].m;
                P->coop_hcap = (int)(ns[0] * small_hplane(ns));
            }
            // per grid level the load vector reduced along dims 2 and 1, then
            // the barrier words
            for (int j = j0; j < s; ++j) {
                const mgard_level &lv = P->lv[j];
                P->coop_g_off.push_back(ws);
                ws = align_up(ws + (size_t)(lv.n[0] * lv.m[1] * lv.m[2]) * P->elem_ws);
            }
            P->coop_bar_off = ws;
            ws = align_up(ws + kMultiBarrierWords * sizeof(unsigned));
            P->ws_bytes = ws;
        } else {
            P->coop_auto = L;
        }
    }
    P->coop_j = P->coop_auto;

    *tab_out = std::move(tab);
    *out = P;
    return MGARD_OK;
}

// Grid of the cooperative kernel: every block resident (both directions), or
// no cooperative kernel when the device cannot hold one block per SM.
template <typename TX, typename TW>
static cudaError_t coop_occupancy(const mgard_plan *P, int *bps)
{
    int a = 0, b = 0;
    cudaError_t err = multi_occupancy<TX, TW>(MODE_DEC, P->coop_smem, &a);
    if (err == cudaSuccess) err = multi_occupancy<TX, TW>(MODE_REC, P->coop_smem, &b);
    *bps = std::min(a, b);
    return err;
}

static cudaError_t configure_coop(mgard_plan *P)
{
    if (P->coop_auto >= P->L) return cudaSuccess;
    int coop_ok = 0;
    cudaError_t err = cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, P->device);
    if (err != cudaSuccess) return err;
    int bps = 0;
    if (coop_ok) {
        const bool user = P->coop_auto == 0;
        switch (P->dtype) {
        case MGARD_F32: err = coop_occupancy<float, float>(P, &bps); break;
        case MGARD_F64: err = coop_occupancy<double, double>(P, &bps); break;
        default: err = user ? coop_occupancy<float, double>(P, &bps) : coop_occupancy<double, double>(P, &bps); break;
        }
        if (err != cudaSuccess) return err;
    }
    if (bps < 1) {
        P->coop_auto = P->coop_j = P->L;
        return cudaSuccess;
    }
    P->coop_grid = bps * P->num_sms;
    return cudaSuccess;
}

// Launch configuration of every level (needs the device, allocates nothing).
static cudaError_t configure_plan(mgard_plan *P)
{
    cudaError_t err = cudaSuccess;
    for (int j = 0; j < P->L && err == cudaSuccess; ++j) {
        mgard_level &lv = P->lv[j];
        switch (P->dtype) {
        case MGARD_F32: err = configure_level<float, float>(P, lv, j == 0); break;
        case MGARD_F64: err = configure_level<double, double>(P, lv, j == 0); break;
        default: err = configure_level<float, double>(P, lv, j == 0); break;
        }
        if (err != cudaSuccess) break;
        switch (P->dtype) {
        case MGARD_F32: err = configure_rc<float, float>(P, lv, j == 0); break;
        case MGARD_F64: err = configure_rc<double, double>(P, lv, j == 0); break;
        default: err = configure_rc<float, double>(P, lv, j == 0); break;
        }
        if (err == cudaSuccess) err = (P->dtype == MGARD_F32) ? configure_slab<float>(P, lv, j == 0)
                                                              : configure_slab<double>(P, lv, j == 0);
    }
    if (err == cudaSuccess) err = configure_coop(P);
    return err;
}

// Slab configuration of every level again (after a tuning change).
static cudaError_t configure_plan_slab(mgard_plan *P)
{
    cudaError_t err = cudaSuccess;
    for (int j = 0; j < P->L && err == cudaSuccess; ++j)
        err = (P->dtype == MGARD_F32) ? configure_slab<float>(P, P->lv[j], j == 0)
                                      : configure_slab<double>(P, P->lv[j], j == 0);
    return err;
}

// Row-chunk configuration of every level again (after a tuning change).
static cudaError_t configure_plan_rc(mgard_plan *P)
{
    cudaError_t err = cudaSuccess;
    for (int j = 0; j < P->L && err == cudaSuccess; ++j) {
        switch (P->dtype) {
        case MGARD_F32: err = configure_rc<float, float>(P, P->lv[j], j == 0); break;
        case MGARD_F64: err = configure_rc<double, double>(P, P->lv[j], j == 0); break;
        default: err = configure_rc<float, double>(P, P->lv[j], j == 0); break;
        }
    }
    return err;
}

// Bytes of the device tables of a plan built by build_plan_host: the double
// tables, then the float tables, 256-byte aligned.
static size_t table_bytes(const std::vector<double> &tab)
{
    return align_up(tab.size() * sizeof(double)) + align_up(tab.size() * sizeof(float));
}

// A uniform-grid plan whose tables live in caller-provided device memory
// `dev` (256-byte aligned, `dev_bytes` long), copied there on `stream`; the
// plan does not own (or free) them.  Fails with MGARD_ERR_WORKSPACE, before
// touching the device, unless the tables (*used bytes) and the plan's
// workspace after them both fit.  Used by the entry point that must not
// allocate.
mgard_status mg_plan_in_place(int ndim, const int64_t *dims, int nlevels, mgard_dtype dtype, void *dev,
                              size_t dev_bytes, cudaStream_t stream, mgard_plan **out, size_t *used)
{
    std::vector<double> tab;
    mgard_plan *P = nullptr;
    mgard_status s = build_plan_host(ndim, dims, nlevels, nullptr, dtype, &P, &tab);
    if (s != MGARD_OK) return s;
    *used = table_bytes(tab);
    if (*used + P->ws_bytes > dev_bytes) {
        const std::string need = std::to_string(*used + P->ws_bytes);
        delete P;
        return fail(MGARD_ERR_WORKSPACE, "this shape needs " + need + " bytes of scratch (tables and workspace); the static scratch holds " +
                                             std::to_string(dev_bytes));
    }
    std::vector<float> tab32(tab.begin(), tab.end());
    P->tab64 = static_cast<double *>(dev);
    P->tab32 = reinterpret_cast<float *>(static_cast<char *>(dev) + align_up(tab.size() * sizeof(double)));
    P->owns_tables = false;
    // pageable host sources: each copy has consumed its buffer when it returns
    cudaError_t err = cudaMemcpyAsync(P->tab64, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(P->tab32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
    // not the slab kernel: its copy-wait status word would need an allocation
    P->slab_off = true;
    if (err == cudaSuccess) err = configure_plan(P);
    if (err != cudaSuccess) {
        delete P;
        return cuda_fail(err, "static plan");
    }
    // no cooperative kernel: its grid-barrier waits report a timeout through
    // the plan's workspace, which does not outlive this call
    P->coop_off = true;
    P->coop_j = P->L;
    *out = P;
    return MGARD_OK;
}

// Decomposition with a host-built plan (used by the entry point that must not
// allocate; validation as in mgard_decompose).
mgard_status mg_decompose_with(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st);

namespace mg {

bool plan_view(const mgard_plan *P, PlanView *v, PlanLevelView *lv)
{
    if (!P || !v) return false;
    v->ndim = P->ndim;
    v->L = P->L;
    v->dtype = P->dtype;
    v->device = P->device;
    v->num_sms = P->num_sms;
    v->elem_user = P->elem_user;
    v->elem_ws = P->elem_ws;
    for (int d = 0; d < 3; ++d) v->n[d] = P->n[d];
    if (lv) {
        const bool f32 = P->elem_ws == sizeof(float);
        for (int j = 0; j < P->L; ++j) {
            const mgard_level &L = P->lv[j];
            for (int d = 0; d < 3; ++d) {
                lv[j].n[d] = L.n[d];
                lv[j].m[d] = L.m[d];
                lv[j].co[d] = L.co[d];
                lv[j].w[d] = f32 ? (const void *)tab_ptr<float>(P, L.w_off[d]) : (const void *)tab_ptr<double>(P, L.w_off[d]);
                lv[j].k[d] = f32 ? (const void *)tab_ptr<float>(P, L.k_off[d]) : (const void *)tab_ptr<double>(P, L.k_off[d]);
                lv[j].fac[d] = f32 ? (const void *)tab_ptr<float>(P, L.t_off[d]) : (const void *)tab_ptr<double>(P, L.t_off[d]);
            }
        }
    }
    return true;
}

}  // namespace mg

extern "C" {

static mgard_status plan_create(int ndim, const int64_t *dims, int nlevels, const double *const *coords,
                                mgard_dtype dtype, mgard_plan **out, const int *dim_levels)
{
    if (!out) return fail(MGARD_ERR_INVALID_ARG, "plan_create: out is NULL");
    *out = nullptr;  // NULL on every failure path
    std::vector<double> tab;
    mgard_plan *P = nullptr;
    mgard_status s = build_plan_host(ndim, dims, nlevels, coords, dtype, &P, &tab, dim_levels);
    if (s != MGARD_OK) return s;
    // device tables in double and float
    std::vector<float> tab32(tab.begin(), tab.end());
    cudaError_t err = cudaMalloc(&P->tab64, tab.size() * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&P->tab32, tab32.size() * sizeof(float));
    if (err == cudaSuccess) err = cudaMemcpy(P->tab64, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(P->tab32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMalloc(&P->d_status, sizeof(unsigned));
    if (err == cudaSuccess) err = cudaMemset(P->d_status, 0, sizeof(unsigned));
    if (err == cudaSuccess && !P->per_dim) err = configure_plan(P);
    if (err != cudaSuccess) {
        mgard_plan_destroy(P);
        return cuda_fail(err, "plan_create: device tables");
    }
    if (P->per_dim) {
        // the persistent kernel runs the plan: a batch of this one field
        s = mgard_batch_create(1, &P, 1, &P->pd_batch);
        if (s == MGARD_OK && mgard_batch_get(P->pd_batch, 0) != 1)
            s = fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_create_per_dim: the shape does not fit the persistent kernel "
                                                  "(rows of at most 1025 nodes, coarse planes within a block's "
                                                  "shared memory)");
        if (s != MGARD_OK) {
            mgard_plan_destroy(P);
            return s;
        }
        P->ws_bytes = std::max(P->ws_bytes, mgard_batch_workspace_bytes(P->pd_batch));
    }
    *out = P;
    return MGARD_OK;
}

mgard_status mgard_plan_create(int ndim, const int64_t *dims, int nlevels, const double *const *coords,
                               mgard_dtype dtype, mgard_plan **out)
{
    return plan_create(ndim, dims, nlevels, coords, dtype, out, nullptr);
}

mgard_status mgard_plan_create_per_dim(int ndim, const int64_t *dims, const int *levels, const double *const *coords,
                                       mgard_dtype dtype, mgard_plan **out)
{
    if (!dims && out) *out = nullptr;
    std::vector<int> all(ndim > 0 && ndim <= 3 ? ndim : 1, -1);
    return plan_create(ndim, dims, -1, coords, dtype, out, levels ? levels : all.data());
}

mgard_status mgard_plan_destroy(mgard_plan *P)
{
    if (!P) return MGARD_OK;
    if (P->pd_batch) mgard_batch_destroy(P->pd_batch);
    if (P->owns_tables) {
        if (P->tab64) cudaFree(P->tab64);
        if (P->tab32) cudaFree(P->tab32);
    }
    if (P->d_status) cudaFree(P->d_status);
    for (auto &r : P->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : P->prof_pool) cudaEventDestroy(e);
    delete P;
    return MGARD_OK;
}

int mgard_plan_levels(const mgard_plan *P) { return P ? P->L : -1; }

size_t mgard_workspace_bytes(const mgard_plan *P) { return P ? P->ws_bytes : 0; }

int mgard_plan_launches(const mgard_plan *P, int recompose)
{
    if (!P) return -1;
    if (P->per_dim) return 1;  // one persistent launch
    // per level: one restriction + ndim solve sweeps (one fewer where the
    // row-chunk restriction solves along dim 2) + the element-wise
    // kernel(s): interpolation (recompose) or coefficients + coarse
    // placement; then one launch for the coarse levels.  Counted for a
    // 16-byte aligned user array.
    const int tail = recompose ? 1 : 2;
    const bool coop = P->coop_j < P->L;
    const int J = coop ? P->coop_j : P->small_j;
    int n = 0;
    for (int j = 0; j < J; ++j) {
        const bool xs = P->lv[j].slab_ty > 0 ? P->lv[j].slab_xs
                                             : P->lv[j].rc_q[0] > 0 && !(P->rc_off & 2) && P->lv[j].rc_xs;
        n += 1 + P->ndim - (xs ? 1 : 0) + tail;
    }
    return n + (J < P->L ? 1 : 0);
}

static mgard_status check_call(const mgard_plan *P, void *data, void *ws, size_t ws_bytes)
{
    if (!P) return fail(MGARD_ERR_INVALID_ARG, "plan is NULL");
    if (!data) return fail(MGARD_ERR_INVALID_ARG, "d_data is NULL");
    if (P->ws_bytes > 0) {
        if (!ws) return fail(MGARD_ERR_WORKSPACE, "d_ws is NULL");
        if (ws_bytes < P->ws_bytes)
            return fail(MGARD_ERR_WORKSPACE, "workspace too small: need " + std::to_string(P->ws_bytes) +
                                                 " bytes, got " + std::to_string(ws_bytes));
        if (reinterpret_cast<uintptr_t>(ws) % kAlign != 0)
            return fail(MGARD_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    }
    if (reinterpret_cast<uintptr_t>(data) % P->elem_user != 0)
        return fail(MGARD_ERR_INVALID_ARG, "d_data is not aligned to its element size");
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
    if (dev != P->device) return fail(MGARD_ERR_INVALID_ARG, "the plan was created on another device");
    return MGARD_OK;
}

}  // extern "C"

mgard_status mg_decompose_with(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st)
{
    return mgard_decompose(P, d_data, d_ws, ws_bytes, st);
}

// Quantization / de-quantization of a plan's field (quant.cuh); mode 0 quantizes
// field -> codes, 1 de-quantizes codes -> field.
template <typename T>
static mgard_status run_quant(const mgard_plan *P, int mode, const double *bins, const void *field,
                              const int32_t *codes_in, void *field_out, int32_t *codes_out, cudaStream_t st)
{
    QuantParams<T> p{};
    p.c = static_cast<const T *>(field);
    p.q = codes_out;
    p.qi = codes_in;
    p.d = static_cast<T *>(field_out);
    p.n0 = P->n[0];
    p.n1 = P->n[1];
    p.n2 = P->n[2];
    p.L = P->L;
    for (int k = 0; k <= P->L; ++k) {
        if (!(bins[k] > 0.0) || !std::isfinite(bins[k]))
            return fail(MGARD_ERR_INVALID_ARG, "quantize: every bin must be positive and finite");
        const T b = static_cast<T>(bins[k]);
        if (!(b > T(0)) || !std::isfinite((double)b))
            return fail(MGARD_ERR_INVALID_ARG, "quantize: a bin is out of the field precision's range");
        p.bin[k] = b;
        p.inv[k] = T(1) / b;
    }
    const int64_t rows = p.n0 * p.n1;
    const int64_t blocks = std::min<int64_t>((rows + kQuantWarps - 1) / kQuantWarps, (int64_t)P->num_sms * 16);
    if (mode == 0) k_quant<T, 0><<<(unsigned)blocks, 32 * kQuantWarps, 0, st>>>(p);
    else k_quant<T, 1><<<(unsigned)blocks, 32 * kQuantWarps, 0, st>>>(p);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? MGARD_OK : cuda_fail(err, mode == 0 ? "quantize kernel" : "dequantize kernel");
}

static mgard_status quant_call(const mgard_plan *P, int mode, const double *bins, const void *field,
                               const int32_t *codes_in, void *field_out, int32_t *codes_out, void *stream)
{
    if (!P) return fail(MGARD_ERR_INVALID_ARG, "quantize: plan is NULL");
    if (P->per_dim) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "quantize: not for per-dimension level counts");
    if (!bins) return fail(MGARD_ERR_INVALID_ARG, "quantize: bins is NULL");
    if (mode == 0 && (!field || !codes_out)) return fail(MGARD_ERR_INVALID_ARG, "quantize: NULL device pointer");
    if (mode == 1 && (!codes_in || !field_out)) return fail(MGARD_ERR_INVALID_ARG, "dequantize: NULL device pointer");
    if (P->L + 1 > kQuantMaxClasses) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "quantize: too many levels");
    const void *f = mode == 0 ? field : field_out;
    if (reinterpret_cast<uintptr_t>(f) % P->elem_user != 0)
        return fail(MGARD_ERR_INVALID_ARG, "quantize: the field is not aligned to its element size");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P->elem_user == 8) return run_quant<double>(P, mode, bins, field, codes_in, field_out, codes_out, st);
    return run_quant<float>(P, mode, bins, field, codes_in, field_out, codes_out, st);
}

// Decomposition (dir 0) or recomposition (dir 1); allow_coop = false keeps
// the cooperative kernel out (batches run fields concurrently on several
// streams, and a cooperative launch holds every SM).
mgard_status mg_transform(const mgard_plan *P, int dir, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st,
                          bool allow_coop)
{
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    if (P->per_dim) {
        void *data[1] = {d_data};
        return dir == 0 ? mgard_batch_decompose(P->pd_batch, data, d_ws, ws_bytes, st)
                        : mgard_batch_recompose(P->pd_batch, data, d_ws, ws_bytes, st);
    }
    char *ws = static_cast<char *>(d_ws);
    if (dir == 0) {
        switch (P->dtype) {
        case MGARD_F32: return exec_decompose<float, float>(P, d_data, ws, st, allow_coop);
        case MGARD_F64: return exec_decompose<double, double>(P, d_data, ws, st, allow_coop);
        default: return exec_decompose<float, double>(P, d_data, ws, st, allow_coop);
        }
    }
    switch (P->dtype) {
    case MGARD_F32: return exec_recompose<float, float>(P, d_data, ws, st, allow_coop);
    case MGARD_F64: return exec_recompose<double, double>(P, d_data, ws, st, allow_coop);
    default: return exec_recompose<float, double>(P, d_data, ws, st, allow_coop);
    }
}

extern "C" {

mgard_status mgard_decompose(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    return mg_transform(P, 0, d_data, d_ws, ws_bytes, static_cast<cudaStream_t>(stream), true);
}

mgard_status mgard_recompose(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    return mg_transform(P, 1, d_data, d_ws, ws_bytes, static_cast<cudaStream_t>(stream), true);
}

mgard_status mgard_recompose_classes(const mgard_plan *P, int nclasses, void *d_data, void *d_ws, size_t ws_bytes,
                                     void *stream)
{
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    if (P->per_dim) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "recompose_classes: not for per-dimension level counts");
    if (nclasses < 1 || nclasses > P->L + 1)
        return fail(MGARD_ERR_INVALID_ARG, "recompose_classes: nclasses must be in 1.." + std::to_string(P->L + 1));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_ws);
    const int D = P->L + 1 - nclasses;
    switch (P->dtype) {
    case MGARD_F32: return exec_recompose_classes<float, float>(P, d_data, ws, st, D);
    case MGARD_F64: return exec_recompose_classes<double, double>(P, d_data, ws, st, D);
    default: return exec_recompose_classes<float, double>(P, d_data, ws, st, D);
    }
}

mgard_status mgard_decompose_adjoint(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    if (P->per_dim) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "decompose_adjoint: not for per-dimension level counts");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_ws);
    switch (P->dtype) {
    case MGARD_F32: return exec_decompose_adjoint<float, float>(P, d_data, ws, st);
    case MGARD_F64: return exec_decompose_adjoint<double, double>(P, d_data, ws, st);
    default: return exec_decompose_adjoint<float, double>(P, d_data, ws, st);
    }
}

mgard_status mgard_recompose_adjoint(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    if (P->per_dim) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "recompose_adjoint: not for per-dimension level counts");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_ws);
    switch (P->dtype) {
    case MGARD_F32: return exec_recompose_adjoint<float, float>(P, d_data, ws, st);
    case MGARD_F64: return exec_recompose_adjoint<double, double>(P, d_data, ws, st);
    default: return exec_recompose_adjoint<float, double>(P, d_data, ws, st);
    }
}

static cudaError_t reconfigure(mgard_plan *P, int j)
{
    switch (P->dtype) {
    case MGARD_F32: return configure_level<float, float>(P, P->lv[j], j == 0);
    case MGARD_F64: return configure_level<double, double>(P, P->lv[j], j == 0);
    default: return configure_level<float, double>(P, P->lv[j], j == 0);
    }
}

mgard_status mgard_plan_tune(mgard_plan *P, int level, int param, int value)
{
    if (!P || level < 0 || level >= P->L) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: bad plan or level");
    if (P->per_dim) return fail(MGARD_ERR_UNSUPPORTED_SHAPE, "plan_tune: not for per-dimension level counts");
    mgard_level &L = P->lv[level];
    const mgard_level saved = L;
    switch (param) {
    case 0:
        if (value < 0 || value >= kRestrictConfigs) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: tile config");
        L.rcfg = value;
        L.rcfg_user = true;
        break;
    case 1:
        if (value < -1 || value > 32) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: solve warps");
        L.svar = value;
        return MGARD_OK;
    case 2:
        if (value < 0) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: chunk planes");
        L.zreq = value;
        break;
    case 3:
        if (value != 0 && value != 1) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: single-block switch");
        P->small_j = value ? P->L : P->small_auto;
        P->coop_j = (value || P->coop_off) ? P->L : P->coop_auto;
        adj_select(P);
        return MGARD_OK;
    case 6:
        if (value < 0) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: barrier poll limit");
        P->coop_spin = value;
        return MGARD_OK;
    case 7:
        if (value < 0 || value > 3) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: row-chunk switch");
        P->rc_off = value;
        return MGARD_OK;
    case 9: {
        if (value < 0) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: row-chunk planes per item");
        P->rc_zreq = value;
        cudaError_t e2 = configure_plan_rc(P);
        if (e2 != cudaSuccess) return cuda_fail(e2, "plan_tune: row-chunk configuration");
        return MGARD_OK;
    }
    case 10:
    case 11:
    case 12:
    case 13:
    case 15:
    case 16: {
        if (param == 10) {
            if (value != 0 && value != 1) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab switch");
            P->slab_off = value != 0;
        } else if (param == 11) {
            if (value < 0) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab planes per chunk");
            L.slab_zreq = value;
        } else if (param == 12) {
            if (value != 0 && value != 4 && value != 6 && value != 8)
                return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab band rows");
            P->slab_tyreq = value;
        } else if (param == 15) {
            if (value != 0 && value != 2 && value != 3) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab blocks per SM");
            P->slab_mbreq = value;
        } else if (param == 16) {
            if (value != 0 && value != 1) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab dim-2 solve switch");
            P->slab_xs_on = value != 0;
        } else {
            if (value != 0 && (value < 2 || value > kSlabMaxSlots))
                return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab ring slots");
            P->slab_nsreq = value;
        }
        cudaError_t e2 = configure_plan_slab(P);
        if (e2 != cudaSuccess) return cuda_fail(e2, "plan_tune: slab configuration");
        return MGARD_OK;
    }
    case 14:
        if (value < 0) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: slab wait hook");
        P->slab_hook = value > 0 ? 1 : 0;
        P->slab_wait_ns = value > 0 ? (unsigned long long)value * 1000ull : 2000000000ull;
        return MGARD_OK;
    case 4:
        if (value != 0 && value != 1) return fail(MGARD_ERR_INVALID_ARG, "plan_tune: cooperative switch");
        P->coop_off = value != 0;
        P->coop_j = (P->coop_off || P->small_j == P->L) ? P->L : P->coop_auto;
        return MGARD_OK;
    default: return fail(MGARD_ERR_INVALID_ARG, "plan_tune: unknown parameter");
    }
    cudaError_t err = reconfigure(P, level);
    if (err != cudaSuccess) {
        L = saved;  // keep the previous, working configuration
        cudaGetLastError();
        return cuda_fail(err, "plan_tune: configuration not supported on this device");
    }
    return MGARD_OK;
}

int mgard_plan_get_tune(const mgard_plan *P, int level, int param)
{
    if (!P || level < 0 || level >= P->L) return -1;
    const mgard_level &L = P->lv[level];
    switch (param) {
    case 0: return L.rcfg;
    case 1: return L.svar;
    case 2: return L.zchunk;
    case 3: return P->small_j == P->L ? 1 : 0;
    case 4: return P->coop_off ? 1 : 0;
    case 5: return P->coop_j < P->L ? P->coop_j : -1;
    case 6: return P->coop_spin;
    case 7: return P->rc_off;
    case 9: return P->rc_zreq;
    case 8: return L.rc_q[1] > 0 ? 32 * (16 / (int)(level == 0 ? P->elem_user : P->elem_ws)) * L.rc_q[1] : 0;
    case 10: return P->slab_off ? 1 : 0;
    case 11: return L.slab_ty > 0 ? L.slab_zc : 0;
    case 12: return L.slab_ty;
    case 13: return L.slab_ty > 0 ? L.slab_ns : 0;
    case 14: return P->slab_hook ? (int)(P->slab_wait_ns / 1000ull) : 0;
    case 15: return L.slab_ty > 0 ? L.slab_mb : 0;
    case 16: return L.slab_ty > 0 ? (L.slab_xs ? 1 : 0) : (P->slab_xs_on ? 1 : 0);
    default: return -1;
    }
}

mgard_status mgard_plan_check(const mgard_plan *P, const void *d_ws, void *stream)
{
    if (!P) return fail(MGARD_ERR_INVALID_ARG, "plan_check: plan is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the slab kernel's sticky copy-wait word (read and cleared)
    if (P->d_status) {
        unsigned sw = 0;
        cudaError_t err = cudaMemcpyAsync(&sw, P->d_status, sizeof(sw), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err == cudaSuccess && sw != 0) err = cudaMemsetAsync(P->d_status, 0, sizeof(unsigned), st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return cuda_fail(err, "plan_check");
        if (sw != 0) return fail(MGARD_ERR_TIMEOUT, "a copy wait of the slab load-vector kernel ran out");
    }
    // the grid-barrier word, when the plan runs the cooperative kernel (its
    // launch clears the word; otherwise the workspace holds anything)
    if (P->coop_j >= P->L) return MGARD_OK;
    if (!d_ws) return fail(MGARD_ERR_INVALID_ARG, "plan_check: d_ws is NULL");
    unsigned word = 0;
    const char *src = static_cast<const char *>(d_ws) + P->coop_bar_off + 2 * sizeof(unsigned);
    cudaError_t err = cudaMemcpyAsync(&word, src, sizeof(word), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "plan_check");
    if (word != 0) return fail(MGARD_ERR_TIMEOUT, "a grid-barrier wait of the cooperative kernel ran out");
    return MGARD_OK;
}

static mgard_status host_call(bool DEC, const mgard_plan *P, const void *h_in, void *h_out, void *d_data,
                              void *d_ws, size_t ws_bytes, void *stream)
{
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    if (!h_in || !h_out) return fail(MGARD_ERR_INVALID_ARG, "host buffer is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)count(P->n) * P->elem_user;
    cudaError_t err = cudaMemcpyAsync(d_data, h_in, bytes, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return cuda_fail(err, "host-to-device copy");
    s = DEC ? mgard_decompose(P, d_data, d_ws, ws_bytes, stream) : mgard_recompose(P, d_data, d_ws, ws_bytes, stream);
    if (s != MGARD_OK) return s;
    err = cudaMemcpyAsync(h_out, d_data, bytes, cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) return cuda_fail(err, "device-to-host copy");
    return MGARD_OK;
}

mgard_status mgard_decompose_host(const mgard_plan *P, const void *h_in, void *h_out, void *d_data, void *d_ws,
                                  size_t ws_bytes, void *stream)
{
    return host_call(true, P, h_in, h_out, d_data, d_ws, ws_bytes, stream);
}

mgard_status mgard_recompose_host(const mgard_plan *P, const void *h_in, void *h_out, void *d_data, void *d_ws,
                                  size_t ws_bytes, void *stream)
{
    return host_call(false, P, h_in, h_out, d_data, d_ws, ws_bytes, stream);
}

mgard_status mgard_quantize(const mgard_plan *P, const double *bins, const void *d_data, int32_t *d_codes, void *stream)
{
    return quant_call(P, 0, bins, d_data, nullptr, nullptr, d_codes, stream);
}

mgard_status mgard_dequantize(const mgard_plan *P, const double *bins, const int32_t *d_codes, void *d_data,
                              void *stream)
{
    return quant_call(P, 1, bins, nullptr, d_codes, d_data, nullptr, stream);
}

mgard_status mgard_decompose_quantize(const mgard_plan *P, const double *bins, void *d_data, int32_t *d_codes,
                                      void *d_ws, size_t ws_bytes, void *stream)
{
    if (!P || !bins || !d_codes) return fail(MGARD_ERR_INVALID_ARG, "decompose_quantize: NULL argument");
    mgard_status s = mgard_decompose(P, d_data, d_ws, ws_bytes, stream);
    if (s != MGARD_OK) return s;
    return mgard_quantize(P, bins, d_data, d_codes, stream);
}

mgard_status mgard_dequantize_recompose(const mgard_plan *P, const double *bins, const int32_t *d_codes,
                                        void *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    if (!P || !bins || !d_codes) return fail(MGARD_ERR_INVALID_ARG, "dequantize_recompose: NULL argument");
    mgard_status s = check_call(P, d_data, d_ws, ws_bytes);
    if (s != MGARD_OK) return s;
    s = mgard_dequantize(P, bins, d_codes, d_data, stream);
    if (s != MGARD_OK) return s;
    return mgard_recompose(P, d_data, d_ws, ws_bytes, stream);
}

mgard_status mgard_profile_enable(mgard_plan *P, int levels)
{
    if (!P || levels < 0) return fail(MGARD_ERR_INVALID_ARG, "profile_enable: bad arguments");
    P->prof_levels = levels;
    return MGARD_OK;
}

int mgard_profile_read(mgard_plan *P, int cap, int *kinds, int *levels_out, int *launches, double *ms)
{
    if (!P || cap < 0) return -1;
    struct Acc {
        int kind, level, count;
        double ms;
    };
    std::vector<Acc> acc;
    int rc = 0;
    for (auto &r : P->prof_pending) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) rc = -1;
        bool found = false;
        for (auto &a : acc)
            if (a.kind == r.kind && a.level == r.level) {
                a.count++;
                a.ms += t;
                found = true;
            }
        if (!found) acc.push_back({r.kind, r.level, 1, (double)t});
        P->prof_pool.push_back(r.a);
        P->prof_pool.push_back(r.b);
    }
    P->prof_pending.clear();
    if (rc != 0) {
        g_last_error = "profile_read: event query failed";
        return -1;
    }
    int n = 0;
    for (auto &a : acc) {
        if (n >= cap) break;
        if (kinds) kinds[n] = a.kind;
        if (levels_out) levels_out[n] = a.level;
        if (launches) launches[n] = a.count;
        if (ms) ms[n] = a.ms;
        ++n;
    }
    return n;
}

}  // extern "C"
