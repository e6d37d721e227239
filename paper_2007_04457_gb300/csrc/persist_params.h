// persist_params.h -- parameters of the persistent batch kernel
// (persist.cuh): many independent fields refactored by one launch whose
// blocks pull work items from a queue.  Internal to the library.
#pragma once

#include <cstdint>

#include "small_params.h"

namespace mg {

constexpr int kPersistThreads = 256;
constexpr int kPersistWarps = kPersistThreads / 32;
// longest fine row (dim 2) a field may have: one row per warp in shared memory
constexpr int64_t kPersistMaxRow = 1025;
// ring of partly reduced rows in phase A: fine rows kept per block
constexpr int kPersistRing = 32;
// columns of a phase-C panel: one line per lane
constexpr int kPersistPanel = 32;
// coarse rows per item of the final placement (eight per warp)
constexpr int kPersistPlaceRows = 64;
// rows of G kept per block in phase C (a ring: the rows of the coarse
// planes two groups of eight ahead are copied while the current ones are
// reduced)
constexpr int kPersistGRing = 128;
constexpr int kPersistSpinLimit = 1 << 22;  // dependency polls (tens of ns each)
// the small tail: arrays of at most this many nodes, finished by one block
constexpr int64_t kPersistSmallNodes = 1000;
constexpr int64_t kPersistSmallBytes = 100 * 1024;

enum PersistKind {
    PK_A = 0,      // fine planes: coefficients (decomposition), coarse gather, G = (K_1 (x) K_2) C
    PK_B = 1,      // coarse planes: solves along dims 2 and 1, then V += z or z into F
    PK_C = 2,      // panels of dim-0 lines: F = K_0 G, then the solve along dim 0
    PK_D = 3,      // fine planes (recomposition): U = C + Pi (V - z)
    PK_SMALL = 4,  // the levels of a small array, one block in shared memory
    PK_PLACE = 5,  // coarse rows of a grid level: final values into its array
};

// One grid level of one field.  Fields with two active dims are relabelled
// (rows, 1, columns), so that their rows are the planes of the items; a
// field's first level works on the user array (type TX), the others on the
// compact coarse array of the level before (type TW).  A dim that does not
// coarsen at the level (co = 0, m = n) has P = I: no interpolation, and its
// stencil factor M and solve with M cancel, so both are skipped.  A level
// whose dim 1 does not coarsen runs "by rows": every fine row is its own
// coarse row, and items take rows instead of planes.
struct PersistLevel {
    void *X;                  // level array
    void *V;                  // compact coarse array V (TW)
    void *F;                  // load vector, then the correction z (TW)
    void *G;                  // load vector with dims 2 and 1 reduced, n0 x m1 x m2 (TW)
    int n[3], m[3];           // fine / coarse node counts (inactive dims = 1)
    const void *w[3];         // interpolation weight pairs (TW)
    const void *k[3];         // 5-point stencil rows (TW)
    const void *fac[3];       // LU factors (a, inv, q) (TW)
    int co[3];                // 1: the dim coarsens at this level (0: inactive, or kept with all its nodes)
    int first;                // 1: X has type TX
};

struct PersistTask {
    int kind;                 // PersistKind
    int level;                // level table index (PK_SMALL: small table index)
    int nlevels;              // PK_PLACE: grid levels from this one to the field's last
    int per;                  // planes per item (PK_A, PK_B, PK_D), coarse rows per item (PK_PLACE)
    int nitems;
    int dep[2];               // tasks every item of which must be done first (-1: none)
};

struct PersistParams {
    const PersistLevel *lv;
    const PersistTask *tasks;
    const int2 *items;        // (task, index within the task), in queue order
    const SmallParams *small;
    int nitems;
    unsigned *next;           // queue head
    unsigned *done;           // per task: items finished
    unsigned *status;         // bit 0: a dependency wait ran out (kept until the host clears it)
    const unsigned *zero;     // a word that stays 0 (the test hook's wait)
    int spin_limit;           // polls before a wait gives up
    int stall;                // test hook: 1 = the first item also waits for a count nothing reaches
    unsigned long long *prof; // measurement (NULL = off): per item kind, ns busy, ns waiting, items
};

constexpr int kPersistKinds = 6;
constexpr int kPersistProfWords = 3 * kPersistKinds;

// Counter words of a launch (reset before it): queue head, the zero word,
// then one per task.
constexpr int kPersistHeadWords = 2;

}  // namespace mg
