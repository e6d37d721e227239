// persist_sched.h -- host side of the persistent batch kernel (persist.cuh):
// the tasks of every level of every field, their dependencies, a cost model
// of their items and the list schedule that orders the device queue.  Host
// code only (no device code), shared by batch.cu and the CPU tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include <vector_functions.h>
#include <vector_types.h>

#include "persist_params.h"
#include "plan_view.h"

namespace mg {

// ---------------------------------------------------------------------------
// Tasks and the list-scheduling model
// ---------------------------------------------------------------------------

struct TaskList {
    std::vector<PersistTask> t;
    std::vector<double> cost;   // ns per item
    std::vector<int> field;
    int add(int kind, int level, int per, int64_t nitems, int d0, int d1, double c, int fld, int nlev = 0)
    {
        PersistTask k;
        k.kind = kind;
        k.level = level;
        k.nlevels = nlev;
        k.per = per;
        k.nitems = (int)nitems;
        k.dep[0] = d0;
        k.dep[1] = d1;
        t.push_back(k);
        cost.push_back(c);
        field.push_back(fld);
        return (int)t.size() - 1;
    }
};

// Cost model of one item (ns): bytes it moves at the per-block share of the
// copy bandwidth (6.8 TB/s over `grid` blocks; reads that the L2 serves at
// twice that), plus a fixed cost per item and the solves' recurrence chains.
struct CostModel {
    double bpn;          // bytes per ns per block
    double over = 1500;  // per item
    size_t eu, ew;
    // rows of an item: a plane's rows (by planes) or `per` rows
    static double rows(const PlanLevelView &l, int per, bool fine) { return l.co[1] ? (double)(fine ? l.n[1] : l.m[1]) : per; }
    double a(const PlanLevelView &l, int per, bool first, bool dec) const
    {
        const double ex = (double)(first ? eu : ew);
        const double fine = rows(l, per, true) * l.n[2] * ex * (dec ? 2.3 : 1.1);
        const double coarse = rows(l, per, false) * l.m[2] * ew * 1.5;
        return over + (fine + coarse) / bpn;
    }
    double c(const PlanLevelView &l) const
    {
        const double bytes = ((double)l.n[0] + l.m[0]) * kPersistPanel * ew;
        return over + bytes / bpn + 60.0 * ((l.m[0] + kPersistWarps - 1) / kPersistWarps);
    }
    double b(const PlanLevelView &l, int per, bool dec) const
    {
        const double bytes = rows(l, per, false) * l.m[2] * ew * (dec ? 3.0 : 2.0);
        return over + bytes / bpn + (l.co[1] ? 30.0 * (l.m[1] + l.m[2]) : 10.0 * l.m[2] / 32 + 300.0);
    }
    double d(const PlanLevelView &l, int per, bool first) const
    {
        const double ex = (double)(first ? eu : ew);
        return over + (rows(l, per, true) * l.n[2] * ex * 2.2 + rows(l, per, false) * l.m[2] * ew * 2.0) / bpn;
    }
    double small() const { return 40000.0; }
    double place(const PlanLevelView &l, bool first) const
    {
        const double rows = std::min<double>(kPersistPlaceRows, (double)l.m[0] * l.m[1]);
        return over + rows * l.m[2] * (double)(ew + 2 * (first ? eu : ew)) / bpn;
    }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Per field, decomposition: per grid level A -> C -> B (B of the level
// before feeds A: its V is the level's array), the small tail, then the
// placement of every grid level.  Recomposition: A of each level after A of
// the level before (it reads the V that one gathered), C -> B per level, the
// small tail after the last A, then D from the coarsest level (after its B
// and the D of the level below it, which completes its V).
template <typename Field>
void build_tasks(const std::vector<Field> &fields, int dir, const CostModel &cm, TaskList &T)
{
    const bool dec = dir == 0;
    for (size_t fi = 0; fi < fields.size(); ++fi) {
        const Field &F = fields[fi];
        const int fld = (int)fi;
        if (F.L == 0) continue;
        // by planes (dim 1 coarsens): one plane per item; by rows: 8 rows
        auto per_of = [](const PlanLevelView &l) { return l.co[1] ? 1 : kPersistWarps; };
        auto fine_units = [](const PlanLevelView &l) { return l.co[1] ? l.n[0] : l.n[0] * l.n[1]; };
        auto coarse_units = [](const PlanLevelView &l) { return l.co[1] ? l.m[0] : l.m[0] * l.m[1]; };
        auto panels = [](const PlanLevelView &l) { return l.m[1] * ceil_div(l.m[2], kPersistPanel); };
        std::vector<int> Bt(F.nd);
        int prev = -1, prevA = -1;
        for (int j = 0; j < F.nd; ++j) {
            const PlanLevelView &l = F.lv[j];
            const int gl = F.lv_base + j, per = per_of(l);
            const int A = T.add(PK_A, gl, per, ceil_div(fine_units(l), per), dec ? prev : prevA, -1,
                                cm.a(l, per, j == 0, dec), fld);
            const int C = T.add(PK_C, gl, 1, panels(l), A, -1, cm.c(l), fld);
            Bt[j] = T.add(PK_B, gl, per, ceil_div(coarse_units(l), per), C, -1, cm.b(l, per, dec), fld);
            prev = Bt[j];
            prevA = A;
        }
        if (dec) {
            if (F.small >= 0) prev = T.add(PK_SMALL, F.small, 1, 1, prev, -1, cm.small(), fld);
            for (int j = 0; j < F.nd; ++j) {
                const PlanLevelView &l = F.lv[j];
                T.add(PK_PLACE, F.lv_base + j, kPersistPlaceRows, ceil_div(l.m[0] * l.m[1], kPersistPlaceRows), prev,
                      -1, cm.place(l, j == 0), fld, F.nd - j);
            }
        } else {
            int last = -1;
            if (F.small >= 0) last = T.add(PK_SMALL, F.small, 1, 1, prevA, -1, cm.small(), fld);
            for (int j = F.nd - 1; j >= 0; --j) {
                const PlanLevelView &l = F.lv[j];
                const int per = per_of(l);
                last = T.add(PK_D, F.lv_base + j, per, ceil_div(fine_units(l), per), Bt[j], last, cm.d(l, per, j == 0),
                             fld);
            }
        }
    }
}

// List schedule of the items on `workers` identical workers: whenever a
// worker is free it takes the next item of the ready task that comes first
// by `prio` (smaller first; ties by task order).  The items in the order
// they were taken form the queue; every item comes after all items of the
// tasks it depends on.  Returns the modelled makespan (ns).
inline double list_schedule(const TaskList &T, const std::vector<int64_t> &prio, int workers, std::vector<int2> &out)
{
    const int nt = (int)T.t.size();
    std::vector<int> ndeps(nt, 0), next(nt, 0), done(nt, 0);
    std::vector<std::vector<int>> users(nt);
    int64_t total = 0;
    for (int i = 0; i < nt; ++i) {
        total += T.t[i].nitems;
        for (int d = 0; d < 2; ++d)
            if (T.t[i].dep[d] >= 0) {
                ++ndeps[i];
                users[T.t[i].dep[d]].push_back(i);
            }
    }
    using Key = std::pair<int64_t, int>;
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> ready;
    auto key = [&](int i) { return Key(prio[i] * (int64_t)nt + i, i); };
    for (int i = 0; i < nt; ++i)
        if (ndeps[i] == 0) ready.push(key(i));
    using Ev = std::pair<double, int>;
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> ev;
    out.clear();
    out.reserve((size_t)total);
    int idle = std::max(1, workers);
    double t = 0, end = 0;
    while ((int64_t)out.size() < total) {
        while (idle > 0 && !ready.empty()) {
            const int i = ready.top().second;
            out.push_back(make_int2(i, next[i]));
            ev.push(Ev(t + T.cost[i], i));
            --idle;
            if (++next[i] == T.t[i].nitems) ready.pop();
        }
        if ((int64_t)out.size() >= total) break;
        if (ev.empty()) return -1.0;  // a dependency that never completes
        const Ev e = ev.top();
        ev.pop();
        t = e.first;
        ++idle;
        if (++done[e.second] == T.t[e.second].nitems)
            for (int u : users[e.second])
                if (--ndeps[u] == 0) ready.push(key(u));
    }
    while (!ev.empty()) {
        end = std::max(end, ev.top().first);
        ev.pop();
    }
    return std::max(end, t);
}

// Every item after all items of its task's dependencies, each exactly once.
inline bool order_ok(const TaskList &T, const std::vector<int2> &items)
{
    const int nt = (int)T.t.size();
    std::vector<int64_t> last(nt, -1), count(nt, 0);
    for (size_t k = 0; k < items.size(); ++k) {
        const int i = items[k].x;
        if (i < 0 || i >= nt || items[k].y != count[i]) return false;
        ++count[i];
        last[i] = (int64_t)k;
    }
    for (int i = 0; i < nt; ++i)
        if (count[i] != T.t[i].nitems) return false;
    for (size_t k = 0; k < items.size(); ++k) {
        const PersistTask &t = T.t[items[k].x];
        for (int d = 0; d < 2; ++d)
            if (t.dep[d] >= 0 && last[t.dep[d]] >= (int64_t)k) return false;
    }
    return true;
}

// Queue priority of every task (smaller first): order 0 = the rank of its
// field (fields by decreasing modelled time: a few fields in flight, their
// levels kept in L2), then task order; order 1 = the longest modelled path
// from the task to the end of its field first (a task's span: its items'
// cost over `grid` workers).  field_rank: rank of every field for order 0.
inline std::vector<int64_t> task_priorities(const TaskList &T, int order, int grid, const std::vector<int> &field_rank)
{
    const int ntk = (int)T.t.size();
    std::vector<int64_t> prio(ntk);
    if (order == 1) {
        std::vector<double> bl(ntk, 0.0);
        for (int i = ntk - 1; i >= 0; --i) {  // dependents come later in the task list
            const double span = T.cost[i] * std::ceil((double)T.t[i].nitems / std::max(1, grid));
            bl[i] += span;
            for (int d = 0; d < 2; ++d)
                if (T.t[i].dep[d] >= 0) bl[T.t[i].dep[d]] = std::max(bl[T.t[i].dep[d]], bl[i]);
        }
        for (int i = 0; i < ntk; ++i) prio[i] = -(int64_t)bl[i];
    } else {
        for (int i = 0; i < ntk; ++i) prio[i] = field_rank[T.field[i]];
    }
    return prio;
}

// Fields by decreasing modelled time (the sum of their items' costs):
// rank[f] = position of field f in that order; nf = number of fields.
inline std::vector<int> field_ranks(const TaskList &T, int nf, std::vector<double> *cost_out = nullptr)
{
    std::vector<double> fc(nf, 0.0);
    for (size_t i = 0; i < T.t.size(); ++i) fc[T.field[i]] += T.cost[i] * T.t[i].nitems;
    std::vector<int> order(nf), rank(nf);
    for (int i = 0; i < nf; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fc[a] > fc[b]; });
    for (int r = 0; r < nf; ++r) rank[order[r]] = r;
    if (cost_out) *cost_out = fc;
    return rank;
}

}  // namespace mg
