// multi_params.h -- parameters of the cooperative kernel that runs the coarse
// end of the hierarchy in one launch (multi.cuh).  Internal to the library.
#pragma once

#include <cstdint>

#include "small_params.h"

namespace mg {

constexpr int kMultiMaxLevels = 8;
constexpr int kMultiThreads = 256;
constexpr int64_t kMultiMaxSide = 129;    // level arrays the grid runs (per side)
// 32-lane chunks of a fine row (<= 129 nodes) and of a coarse row (<= 65)
constexpr int kMultiRowChunks = 5;
constexpr int kMultiCoarseChunks = 3;
// block 0 takes over once the array has at most this many nodes and its
// shared-memory layout (small.cuh, H holding every fine plane) fits
constexpr int64_t kMultiSmallNodes = 1000;
constexpr int64_t kMultiSmallBytes = 100 * 1024;
constexpr int kMultiBarrierWords = 3;
constexpr int kMultiSpinLimit = 1 << 22;  // barrier polls (tens of ns each)
// shared-memory elements for a phase's tables, ahead of its data: weights
// and stencil rows of dims 1 and 2 (<= 2*129 + 2*129 + 5*65 + 5*65), or
// LU factors (<= 3*65 per dim); a multiple of 16 bytes for both types
constexpr int kMultiTabElems = 1280;

struct MultiLevel {
    void *X;                  // level array (type TX for the first level, TW after)
    void *V;                  // compact coarse array V (TW)
    void *F;                  // load vector, then the correction z (TW)
    void *G;                  // load vector with dims 2 and 1 reduced, n0 x m1 x m2 (TW)
    int n[3], m[3];           // fine / coarse node counts (inactive dims = 1)
    const void *w[3];         // interpolation weight pairs (TW)
    const void *k[3];         // 5-point stencil rows (TW)
    const void *fac[3];       // LU factors (a, inv, q) (TW)
};

struct MultiParams {
    MultiLevel lv[kMultiMaxLevels];
    int nd;                   // levels run by the whole grid
    int small;                // 1: block 0 then runs the remaining levels in shared memory
    SmallParams sp;           // those levels (array = V of the last grid level)
    unsigned *bar;            // grid barrier: arrivals, generation, timeout record
    int spin_limit;           // barrier polls before a wait gives up
};

// Shared-memory elements one block needs for a grid level: a fine plane and
// its coarse grid or its dim-2 reduction (n1 x m2), five coarse planes of
// the partly reduced load vector, or two slices of coarse lines along dim 0.
inline int64_t multi_level_elems(const int64_t *n, const int64_t *m)
{
    int64_t a = n[1] * n[2] + (m[1] * m[2] > n[1] * m[2] ? m[1] * m[2] : n[1] * m[2]);
    if (5 * m[1] * m[2] > a) a = 5 * m[1] * m[2];
    if (2 * m[0] * m[2] > a) a = 2 * m[0] * m[2];
    return a;
}

}  // namespace mg
