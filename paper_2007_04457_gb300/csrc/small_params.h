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

// Elements of the tables of nlev levels of an array of n nodes per dim:
// 2 interpolation weights per fine node, 5 stencil entries and 3 LU factors
// per coarse node, for every active dim of every level.
inline int64_t small_tab_elems(const int64_t *n, int nlev)
{
    int64_t t = 0;
    for (int i = 0; i < nlev; ++i)
        for (int k = 0; k < 3; ++k)
            if (n[k] > 1) {
                const int64_t nf = (n[k] - 1) / (int64_t(1) << i) + 1;
                t += 2 * nf + 8 * ((nf - 1) / 2 + 1);
            }
    return t;
}

// Largest dynamic shared memory the single-block kernel asks for, and the
// longest dimension it takes (its solves run one thread per line).
constexpr int64_t kSmallMaxBytes = 227 * 1024;
constexpr int64_t kSmallMaxSide = 257;

}  // namespace mg
