// plan_view.h -- a read-only view of a plan's levels for the batch code
// (batch.cu), which builds its own work lists from them.  Internal.
#pragma once

#include <cstdint>

#include "mgard.h"

namespace mg {

struct PlanLevelView {
    int64_t n[3], m[3];              // fine / coarse node counts (leading dims padded with 1)
    int co[3];                       // 1: the dim coarsens at this level
    const void *w[3], *k[3], *fac[3];  // device tables in the plan's arithmetic type
};

struct PlanView {
    int ndim;                        // squeezed dimension count
    int L;                           // levels
    mgard_dtype dtype;
    int device, num_sms;
    size_t elem_user, elem_ws;       // bytes of a user element / an arithmetic element
    int64_t n[3];                    // finest node counts
};

// Fills *v and, when lv is given, lv[0 .. L-1].  False for a NULL plan.
bool plan_view(const mgard_plan *P, PlanView *v, PlanLevelView *lv);

}  // namespace mg
