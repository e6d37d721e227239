// small_params.h -- parameters of the single-block kernel that runs every
// remaining level of a small array (small.cuh).  Internal to the library.
#pragma once

#include <cstdint>

namespace mg {

constexpr int kSmallMaxLevels = 16;

struct SmallParams {
    void *A;                                 // level array, type T, in place
    int n[3];                                // node counts (inactive dims = 1)
    int nlev;                                // levels run inside the block
    int hcap;                                // elements of the dim-2 scratch H
    const void *w[kSmallMaxLevels][3];       // interpolation weight pairs, type TW
    const void *k[kSmallMaxLevels][3];       // 5-point stencil rows, type TW
    const void *fac[kSmallMaxLevels][3];     // LU factors (a, inv, q), type TW
};

// Shared-memory elements the kernel needs for an array of n nodes per dim
// besides H (the array, G and F).
inline int64_t small_elems(const int64_t *n)
{
    int64_t m[3];
    for (int k = 0; k < 3; ++k) m[k] = (n[k] > 1) ? (n[k] - 1) / 2 + 1 : 1;
    return n[0] * n[1] * n[2] + n[0] * m[1] * m[2] + m[0] * m[1] * m[2];
}

// Elements of one fine plane of H at the first level.
inline int64_t small_hplane(const int64_t *n)
{
    const int64_t m2 = (n[2] > 1) ? (n[2] - 1) / 2 + 1 : 1;
    return n[1] * m2;
}

// Largest dynamic shared memory the single-block kernel asks for, and the
// longest dimension it takes (its solves run one thread per line).
constexpr int64_t kSmallMaxBytes = 227 * 1024;
constexpr int64_t kSmallMaxSide = 257;

}  // namespace mg
