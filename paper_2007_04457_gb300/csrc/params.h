// params.h -- launch parameter blocks passed by value from the host level
// loop to the kernels.  Internal to the library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mg {

// Active-dimension masks: bit 2 = dim 0 (slowest, "z"), bit 1 = dim 1 ("y"),
// bit 0 = dim 2 (contiguous, "x").  1D grids use 1, 2D grids 3, 3D grids 7.
enum : int { ACT_1D = 1, ACT_2D = 3, ACT_3D = 7 };

enum : int { MODE_DEC = 0, MODE_REC = 1 };

// Fused coefficient + load-vector pass over one level array (Section III-A:
// the grid-processing coefficient step and the linear-processing
// mass-transfer stencil, fused into a single tiled sweep).
struct RestrictParams {
    void *A;                 // level array, element type T (in/out)
    void *F;                 // load vector on N_{l-1}, element type TW (out)
    void *V;                 // values of A at N_{l-1}, element type TW (out)
    int64_t n0, n1, n2;      // level-l node counts (inactive dims = 1)
    int64_t m0, m1, m2;      // level-(l-1) node counts
    const void *w0, *w1, *w2;  // interpolation weight pairs per fine node, type T
    const void *k0, *k1, *k2;  // 5-point R*M stencil per coarse node, type T
    int tiles_y, tiles_x;    // tile grid over (dim 1, dim 2) in coarse nodes
    int zchunk, nzc;         // coarse planes per work item, number of chunks
    int nitems;              // tiles_y * tiles_x * nzc
    int kuni1;               // 1: the interior rows of k1 are all equal
};

// Tridiagonal solves along one dimension of a compact coarse array, with the
// LU factors of M_{l-1} precomputed per node: forward y_i = f_i - a_i y_{i-1},
// backward z_i = inv_i y_i - q_i z_{i+1} (Section III-A-3, Thomas algorithm).
struct SolveParams {
    void *F;                 // right-hand sides, solved in place (type TW)
    void *V;                 // coarse values updated by +-z when vmode != 0
    const void *fac;         // 3 factors (a, inv, q) per node along the line
    int64_t nlines;          // number of lines
    int64_t inner;           // product of dims after the solved one
    int64_t stride;          // element stride along the line (= inner)
    int m;                   // line length
    int nw;                  // warps per block (chunks per line)
    int chunk;               // nodes per chunk
    int vmode;               // 0: F <- z, 1: V += z, 2: V -= z
    int lpb;                 // lines per block
    const void *src;         // right-hand sides read from here instead of F (may be null)
};

// Element-wise level kernels: placement of coefficients and coarse values
// after a decomposition level (k_place), and the recomposition of a level
// from its coefficients and the corrected coarse values (k_interp).
struct PlaceParams {
    void *A;                 // level array (type T)
    const void *V;           // compact coarse array (type TW)
    int64_t n0, n1, n2, m0, m1, m2;
    const void *w0, *w1, *w2;  // interpolation weight pairs per fine node, type T
    int64_t zchunk, nzc;     // k_sweep: fine planes per work item (even), chunk count
};

// Transposed level maps (adjoint.cuh).
struct AdjParams {
    void *A;                 // level array (type T)
    const void *Z;           // k_adj_odd: solved coarse array; k_adj_even: compact base or null (type TW)
    int64_t n0, n1, n2, m0, m1, m2;
    const void *k0, *k1, *k2;  // R*M stencil rows, type TW
    const void *w0, *w1, *w2;  // interpolation weight pairs, type T
    int sign;                // +1 or -1
};

// Finest-grid values of a level-k function (prolong.cuh): multilinear
// interpolation of compact level-k values onto every node of the finest grid.
struct ProlongParams {
    void *out;               // finest array (type T), n0 x n1 x n2
    const void *V;           // level-k values (type TW), m0 x m1 x m2
    const void *w0, *w1, *w2;  // per finest node: weight of its right level-k neighbour (TW)
    int n0, n1, n2, m0, m1, m2;
    int shift;               // finest index >> shift = left level-k neighbour (>= 1)
    int seg;                 // launcher only: row segment it sizes the grid by (the
                             // kernel walks its own strips of 32 columns x 64 rows)
};


// Row-chunk level kernels (rowchunk.cuh): a warp takes one segment of 32 C
// fine columns of a row (lane L: columns C L .. C L + C - 1, plus the
// segment's closing column for the last segment), so every row is moved in
// aligned 16-byte words.  Level arrays are 16-byte aligned; n1 - 1 is a
// multiple of 8 and n2 - 1 = 32 C S.
constexpr int kRcWarps = 4;  // warps per block of the row-chunk kernels
// coarse rows per row-chunk restriction item (a kernel template argument:
// this toolkit's device compiler stops on the kernel when it derives the
// count from its other arguments); four rows per item were measured slower
constexpr int kRcRows = 2;
// row-chunk kernels kept out by default (bit 0 sweeps, bit 1 restriction):
// the restriction is measured slower than the strip kernel + dim-2 solve
constexpr int kRcDefaultOff = 2;

struct RcParams {
    void *A;                   // level array (type T), n0 x n1 x n2
    void *F;                   // load vector on N_{l-1} (type TW)
    void *V;                   // coarse values (type TW)
    int n0, n1, n2, m0, m1, m2;
    int S;                     // segments per row
    int nb;                    // row items: coarse rows (sweep) or row blocks (restriction)
    int zchunk, nzc;           // coarse intervals / planes per chunk, chunk count
    int nitems;                // S * nb * nzc
    const void *w0, *w1, *w2;  // interpolation weight pairs per fine node (type T)
    const void *k0, *k1, *k2;  // K = P^T M_l rows, 5 per coarse node (type T)
    const void *fx;            // LU factors of M_{l-1} along dim 2, 3 per coarse node (type TW)
};

// Load vector and coarse gather of a 3D level from whole-row slabs staged in
// shared memory by bulk asynchronous copies (slab.cuh): 4-byte level arrays
// with rows of n2 = 128 k + 1 nodes, one block of (n2 - 1) / 4 threads per
// band of coarse rows x chunk of coarse planes.
struct SlabParams {
    const void *A;             // level array (float), n0 x n1 x n2
    void *F;                   // load vector on N_{l-1} (type TW)
    void *V;                   // values of A at N_{l-1} (type TW)
    int n0, n1, n2, m0, m1, m2;
    const void *k0, *k1, *k2;  // K = P^T M_l rows, 5 per coarse node (float)
    int nb;                    // bands of TY coarse rows (the last shifted back)
    int zchunk, nzc;           // coarse planes per chunk, chunk count
    int nitems;                // nb * nzc
    int ns;                    // ring slots (planes staged at once)
    int slot_bytes;            // bytes per slot, a 16-byte multiple
    int kuni1;                 // 1: the interior rows of k1 are all equal
    int hook;                  // test hook: each block's first copy wait runs out
    unsigned *status;          // sticky status word: bit 0 = a copy wait ran out
    unsigned long long wait_ns;  // limit of one copy wait
    const void *fx;            // LU factors of M_{l-1} along dim 2, 3 per coarse node (type TW)
};

}  // namespace mg
