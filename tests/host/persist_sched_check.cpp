// Checks of the persistent batch kernel's host scheduler (persist_sched.h) on
// synthetic fields, without a GPU: every item is queued exactly once and
// after every item of the tasks it depends on; item counts per task kind
// follow the level geometry; one worker's makespan is the sum of all item
// costs; more workers never take longer than one; a queue with an item moved
// before its dependencies is rejected.  Prints one line per check, exits 1 on
// the first failure.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "persist_sched.h"

using namespace mg;

namespace {

struct Field {
    int L = 0, nd = 0, small = -1, lv_base = 0;
    std::vector<PlanLevelView> lv;
};

int fails = 0;

void check(bool ok, const char *what)
{
    std::printf("%s %s\n", ok ? "ok" : "FAIL", what);
    if (!ok) ++fails;
}

// Levels of a field with fine counts n (leading dims 1 when inactive) and a
// per-dimension level count lk (dimension d coarsens in the first lk[d] steps).
Field make_field(const int64_t n0[3], const int lk[3], int nd, int small, int base)
{
    static const double dummy = 0.0;
    Field F;
    int L = 0;
    for (int d = 0; d < 3; ++d) L = std::max(L, lk[d]);
    F.L = L;
    F.nd = nd;
    F.small = small;
    F.lv_base = base;
    int64_t n[3] = {n0[0], n0[1], n0[2]};
    for (int j = 0; j < L; ++j) {
        PlanLevelView v{};
        for (int d = 0; d < 3; ++d) {
            v.n[d] = n[d];
            v.co[d] = (n[d] > 1 && j < lk[d]) ? 1 : 0;
            v.m[d] = v.co[d] ? (n[d] - 1) / 2 + 1 : n[d];
            v.w[d] = v.k[d] = v.fac[d] = &dummy;
        }
        F.lv.push_back(v);
        for (int d = 0; d < 3; ++d) n[d] = v.m[d];
    }
    return F;
}

int64_t items_of_kind(const TaskList &T, int kind)
{
    int64_t s = 0;
    for (const auto &t : T.t)
        if (t.kind == kind) s += t.nitems;
    return s;
}

}  // namespace

int main()
{
    std::vector<Field> fields;
    int base = 0;
    const int64_t cube[3] = {257, 257, 257}, slab[3] = {17, 65, 129}, rows2d[3] = {1025, 1, 1025};
    const int lcube[3] = {8, 8, 8}, lslab[3] = {4, 4, 4}, l2d[3] = {10, 0, 10}, lper[3] = {2, 6, 3};
    fields.push_back(make_field(cube, lcube, 5, 0, base));      // grid levels 0..4, a small tail
    base += 5;
    fields.push_back(make_field(slab, lslab, 4, -1, base));     // every level on the grid
    base += 4;
    fields.push_back(make_field(rows2d, l2d, 6, 1, base));      // two active dims, by rows
    base += 6;
    const int64_t pd[3] = {17, 65, 33};
    fields.push_back(make_field(pd, lper, 6, -1, base));        // per-dimension counts
    base += 6;

    for (int dir = 0; dir < 2; ++dir) {
        for (int grid : {1, 7, 304}) {
            CostModel cm;
            cm.bpn = 6800.0 / grid;
            cm.eu = cm.ew = 4;
            TaskList T;
            build_tasks(fields, dir, cm, T);
            const std::vector<int> rank = field_ranks(T, (int)fields.size());
            double serial = 0;
            for (size_t i = 0; i < T.t.size(); ++i) serial += T.cost[i] * T.t[i].nitems;
            for (int order = 0; order < 2; ++order) {
                std::vector<int64_t> prio = task_priorities(T, order, grid, rank);
                std::vector<int2> items;
                const double ms = list_schedule(T, prio, grid, items);
                char what[160];
                std::snprintf(what, sizeof(what), "dir %d grid %d order %d: queue respects dependencies", dir, grid,
                              order);
                check(ms > 0 && order_ok(T, items), what);
                if (grid == 1) {
                    std::snprintf(what, sizeof(what), "dir %d order %d: one worker takes the sum of item costs", dir,
                                  order);
                    check(std::abs(ms - serial) <= 1e-6 * serial, what);
                } else {
                    std::snprintf(what, sizeof(what), "dir %d grid %d order %d: makespan at most the serial time", dir,
                                  grid, order);
                    check(ms <= serial * (1 + 1e-9), what);
                }
                if (!items.empty()) {
                    std::vector<int2> bad = items;
                    std::swap(bad.front(), bad.back());
                    std::snprintf(what, sizeof(what), "dir %d grid %d order %d: a reordered queue is rejected", dir,
                                  grid, order);
                    check(!order_ok(T, bad), what);
                }
            }
            // item counts per kind: planes (or 8-row groups) for A and D,
            // coarse planes (or groups) for B, 32-column panels for C
            int64_t a = 0, b = 0, c = 0, place = 0, small = 0;
            for (const auto &F : fields)
                for (int j = 0; j < F.nd; ++j) {
                    const PlanLevelView &l = F.lv[j];
                    const int per = l.co[1] ? 1 : kPersistWarps;
                    a += ceil_div(l.co[1] ? l.n[0] : l.n[0] * l.n[1], per);
                    b += ceil_div(l.co[1] ? l.m[0] : l.m[0] * l.m[1], per);
                    c += l.m[1] * ceil_div(l.m[2], kPersistPanel);
                    place += ceil_div(l.m[0] * l.m[1], kPersistPlaceRows);
                }
            for (const auto &F : fields) small += F.small >= 0 ? 1 : 0;
            char what[160];
            std::snprintf(what, sizeof(what), "dir %d grid %d: items per kind", dir, grid);
            check(items_of_kind(T, PK_A) == a && items_of_kind(T, PK_B) == b && items_of_kind(T, PK_C) == c &&
                      items_of_kind(T, PK_SMALL) == small &&
                      items_of_kind(T, PK_PLACE) == (dir == 0 ? place : 0) &&
                      items_of_kind(T, PK_D) == (dir == 1 ? a : 0),
                  what);
        }
    }
    std::printf("%s\n", fails ? "FAILED" : "ALL OK");
    return fails ? 1 : 0;
}
