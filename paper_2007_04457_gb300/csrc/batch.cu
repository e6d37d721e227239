// batch.cu -- batches of independent fields.
//
// A batch runs in one of two ways.
//
// Persistent (the default when every field fits it): one launch of the
// persistent kernel (persist.cuh) per direction.  The host cuts every level
// of every field into tasks (A: fine planes, B: coarse planes, C: panels of
// dim-0 lines, D: fine planes of the recomposition, the small tail, the final
// placement), links each task to the tasks it needs, and orders all items by
// a list-scheduling model of the launch: as many workers as the grid has
// blocks, a cost per item from the bytes it moves, and among the ready
// tasks the field with the largest modelled time first, so that a few
// fields at a time are in flight and their levels stay in the L2 cache.  The
// counter reset and the launch are captured in a CUDA graph; the level table
// (data and workspace pointers) is uploaded when the pointers change.
//
// Graph of per-field launches (fields the persistent kernel cannot take,
// or on request): on the first call for a set of pointers the batch
// captures a fork over `streams` internal streams (fields assigned largest
// first to the least loaded stream), each field's level kernels on its
// stream, and the join back; later calls replay the graph.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "launch.cuh"
#include "mgard.h"
#include "persist.cuh"
#include "persist_sched.h"
#include "plan_view.h"

mgard_status mg_fail(mgard_status st, const std::string &msg);
mgard_status mg_cuda_fail(cudaError_t err, const char *what);
mgard_status mg_transform(const mgard_plan *P, int dir, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st,
                          bool allow_coop);

using namespace mg;

namespace {

constexpr size_t kSliceAlign = 256;

size_t align_up(size_t x) { return (x + kSliceAlign - 1) / kSliceAlign * kSliceAlign; }

struct Graph {
    std::vector<void *> data;
    void *ws = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// One field as the persistent kernel sees it: levels relabelled (two active
// dims -> rows, 1, columns), grid levels 0 .. nd-1, the rest in the small tail.
struct PField {
    int L = 0, nd = 0;
    std::vector<PlanLevelView> lv;
    size_t off = 0;                            // first byte of its arrays in the workspace
    std::vector<size_t> v_off, f_off, g_off;   // per grid level, relative to off
    int small = -1;                            // index of its small tail
    int lv_base = 0;                           // its first entry in the level table
    double cost = 0;                           // modelled time of the field alone (ns)
};

struct Persist {
    bool eligible = false;
    std::string why;
    bool on = false;                           // batch calls use the persistent kernel
    mgard_dtype dtype = MGARD_F32;
    size_t eu = 4, ew = 4;                     // bytes of a user / arithmetic element
    std::vector<PField> f;
    std::vector<SmallParams> small_tmpl;       // A filled per call
    int nlevels = 0;
    size_t smem = 0, ws_bytes = 0;
    int num_sms = 0, occupancy = 0, bps_req = 0, grid = 0;
    int spin = kPersistSpinLimit, stall = 0;
    int order = 0;                             // queue order: 0 fields by size, 1 longest remaining path
    std::vector<PersistTask> tasks[2];
    std::vector<int2> items[2];
    double model_ns[2] = {0, 0};
    PersistTask *d_tasks[2] = {nullptr, nullptr};
    int2 *d_items[2] = {nullptr, nullptr};
    PersistLevel *d_lv[2] = {nullptr, nullptr};
    SmallParams *d_small[2] = {nullptr, nullptr};
    unsigned *d_cnt[2] = {nullptr, nullptr};
    unsigned *d_status = nullptr;              // one sticky word per direction
    bool prof_on = false;
    unsigned long long *d_prof = nullptr;      // per direction kPersistProfWords counters
    std::vector<PersistLevel> h_lv[2];
    std::vector<SmallParams> h_small[2];
    std::vector<void *> data[2];
    void *ws[2] = {nullptr, nullptr};
    bool uploaded[2] = {false, false};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
};

}  // namespace

struct mgard_batch {
    std::vector<mgard_plan *> plans;
    std::vector<size_t> offsets;     // workspace slice of each field (graph path)
    std::vector<int> stream_of;      // internal stream of each field
    size_t graph_ws = 0;
    size_t ws_bytes = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // fork event + one join event per stream
    Graph graphs[2];                  // decompose, recompose
    Persist ps;
};

namespace {

int64_t cnt3(const int64_t *n) { return n[0] * n[1] * n[2]; }

// Two active dims (1, r, c) -> (r, 1, c): dim 1's tables move to dim 0.
PlanLevelView relabel(const PlanLevelView &v)
{
    PlanLevelView o = v;
    o.n[0] = v.n[1]; o.m[0] = v.m[1]; o.w[0] = v.w[1]; o.k[0] = v.k[1]; o.fac[0] = v.fac[1]; o.co[0] = v.co[1];
    o.n[1] = 1; o.m[1] = 1; o.w[1] = v.w[0]; o.k[1] = v.k[0]; o.fac[1] = v.fac[0]; o.co[1] = 0;
    return o;
}

// Shared-memory elements the persistent kernel needs for grid level v.
int64_t level_smem_elems(const PlanLevelView &v)
{
    const int n1 = (int)v.n[1], n2 = (int)v.n[2], m0 = (int)v.m[0], m1 = (int)v.m[1], m2 = (int)v.m[2];
    const int pm = v.co[1];
    int64_t e = PersistSmem::a(pm, n1, n2, m1, m2);
    e = std::max<int64_t>(e, PersistSmem::b(pm, m1, m2));
    e = std::max<int64_t>(e, PersistSmem::c(m0));
    e = std::max<int64_t>(e, PersistSmem::d(pm, n1, n2, m2));
    return e;
}

// A dim kept with all its nodes at some level (per-dimension level counts).
bool has_kept_dims(const std::vector<PlanLevelView> &lv)
{
    for (const auto &l : lv)
        for (int d = 0; d < 3; ++d)
            if (l.n[d] > 1 && !l.co[d]) return true;
    return false;
}

constexpr int64_t kPersistMaxSmem = 227 * 1024 - 64;

// Fields, workspace layout and shared memory of the persistent kernel, or
// the reason it cannot take the batch.
bool persist_analyse(const std::vector<mgard_plan *> &plans, Persist &S)
{
    S.f.clear();
    S.small_tmpl.clear();
    S.nlevels = 0;
    int64_t smem_el = 0;
    size_t ws = 0;
    PlanView v0;
    if (!plan_view(plans[0], &v0, nullptr)) {
        S.why = "NULL plan";
        return false;
    }
    S.dtype = v0.dtype;
    S.eu = v0.elem_user;
    S.ew = v0.elem_ws;
    S.num_sms = v0.num_sms;
    for (size_t i = 0; i < plans.size(); ++i) {
        PlanView v;
        plan_view(plans[i], &v, nullptr);
        if (v.dtype != S.dtype || v.device != v0.device) {
            S.why = "fields of different element types or devices";
            return false;
        }
        PField F;
        F.L = v.L;
        F.lv.resize(v.L);
        if (v.L > 0) plan_view(plans[i], &v, F.lv.data());
        if (v.ndim == 2)
            for (auto &l : F.lv) l = relabel(l);
        if (v.L == 0) {
            S.f.push_back(F);
            continue;
        }
        if (F.lv[0].n[2] > kPersistMaxRow) {
            S.why = "a field has rows longer than " + std::to_string(kPersistMaxRow) + " nodes";
            return false;
        }
        // the small tail: from the first level j >= 1 whose array (V_{j-1})
        // is small enough for one block (its levels coarsen every dim)
        F.nd = F.L;
        for (int j = has_kept_dims(F.lv) ? F.L : 1; j < F.L; ++j) {
            const int64_t *ns = F.lv[j - 1].m;
            const int64_t hp = small_hplane(ns), nlev = F.L - j;
            const int64_t el = small_elems(ns) + ns[0] * hp + small_tab_elems(ns, (int)nlev);
            if (cnt3(ns) <= kPersistSmallNodes && el * (int64_t)S.ew <= kPersistSmallBytes &&
                nlev <= kSmallMaxLevels) {
                F.nd = j;
                SmallParams sp;
                std::memset(&sp, 0, sizeof(sp));
                for (int d = 0; d < 3; ++d) sp.n[d] = (int)ns[d];
                sp.nlev = (int)nlev;
                sp.hcap = (int)(ns[0] * hp);
                for (int q = 0; q < sp.nlev; ++q)
                    for (int d = 0; d < 3; ++d) {
                        sp.w[q][d] = F.lv[j + q].w[d];
                        sp.k[q][d] = F.lv[j + q].k[d];
                        sp.fac[q][d] = F.lv[j + q].fac[d];
                    }
                F.small = (int)S.small_tmpl.size();
                S.small_tmpl.push_back(sp);
                smem_el = std::max(smem_el, el);
                break;
            }
        }
        F.off = ws;
        size_t o = 0;
        for (int j = 0; j < F.nd; ++j) {
            const PlanLevelView &l = F.lv[j];
            smem_el = std::max(smem_el, level_smem_elems(l));
            const int64_t mc = cnt3(l.m);
            F.v_off.push_back(o);
            o = align_up(o + (size_t)mc * S.ew);
            F.f_off.push_back(o);
            o = align_up(o + (size_t)mc * S.ew);
            F.g_off.push_back(o);
            o = align_up(o + (size_t)(l.n[0] * l.m[1] * l.m[2]) * S.ew);
        }
        ws += o;
        F.lv_base = S.nlevels;
        S.nlevels += F.nd;
        S.f.push_back(F);
    }
    S.smem = (size_t)smem_el * S.ew;
    if ((int64_t)S.smem > kPersistMaxSmem) {
        S.why = "a level needs more shared memory than a block has";
        return false;
    }
    S.ws_bytes = align_up(ws);
    return true;
}

template <typename TX, typename TW>
cudaError_t occupancy_of(size_t smem, int *bps)
{
    int a = 0, b = 0;
    cudaError_t err = persist_occupancy<TX, TW>(MODE_DEC, smem, &a);
    if (err == cudaSuccess) err = persist_occupancy<TX, TW>(MODE_REC, smem, &b);
    *bps = std::min(a, b);
    return err;
}

cudaError_t persist_occ(const Persist &S, int *bps)
{
    switch (S.dtype) {
    case MGARD_F32: return occupancy_of<float, float>(S.smem, bps);
    case MGARD_F64: return occupancy_of<double, double>(S.smem, bps);
    default: return occupancy_of<float, double>(S.smem, bps);
    }
}

void free_dev(Persist &S, int dir)
{
    cudaFree(S.d_tasks[dir]);
    cudaFree(S.d_items[dir]);
    cudaFree(S.d_lv[dir]);
    cudaFree(S.d_small[dir]);
    cudaFree(S.d_cnt[dir]);
    S.d_tasks[dir] = nullptr;
    S.d_items[dir] = nullptr;
    S.d_lv[dir] = nullptr;
    S.d_small[dir] = nullptr;
    S.d_cnt[dir] = nullptr;
    if (S.exec[dir]) cudaGraphExecDestroy(S.exec[dir]);
    S.exec[dir] = nullptr;
    S.uploaded[dir] = false;
}

// Grid, tasks, queue order and device tables of both directions.
mgard_status persist_build(Persist &S)
{
    int bps = 0;
    cudaError_t err = persist_occ(S, &bps);
    if (err != cudaSuccess) return mg_cuda_fail(err, "batch: occupancy of the persistent kernel");
    if (bps < 1) return mg_fail(MGARD_ERR_INTERNAL, "batch: the persistent kernel does not fit an SM");
    S.occupancy = bps;
    const int use = (S.bps_req > 0) ? std::min(S.bps_req, bps) : bps;
    S.grid = use * S.num_sms;
    CostModel cm;
    cm.bpn = 6800.0 / S.grid;
    cm.eu = S.eu;
    cm.ew = S.ew;
    for (int dir = 0; dir < 2; ++dir) {
        TaskList T;
        build_tasks(S.f, dir, cm, T);
        const int nf = (int)S.f.size();
        std::vector<double> fc;
        const std::vector<int> rank = field_ranks(T, nf, &fc);
        for (int i = 0; i < nf; ++i) S.f[i].cost = fc[i];
        const std::vector<int64_t> prio = task_priorities(T, S.order, S.grid, rank);
        std::vector<int2> items;
        S.model_ns[dir] = list_schedule(T, prio, S.grid, items);
        if (S.model_ns[dir] < 0 || !order_ok(T, items))
            return mg_fail(MGARD_ERR_INTERNAL, "batch: the work list does not respect the task dependencies");
        S.tasks[dir] = T.t;
        S.items[dir] = std::move(items);
        free_dev(S, dir);
        const size_t nt = S.tasks[dir].size(), ni = S.items[dir].size();
        err = cudaMalloc(&S.d_tasks[dir], std::max<size_t>(1, nt) * sizeof(PersistTask));
        if (err == cudaSuccess) err = cudaMalloc(&S.d_items[dir], std::max<size_t>(1, ni) * sizeof(int2));
        if (err == cudaSuccess)
            err = cudaMalloc(&S.d_lv[dir], std::max<size_t>(1, (size_t)S.nlevels) * sizeof(PersistLevel));
        if (err == cudaSuccess)
            err = cudaMalloc(&S.d_small[dir], std::max<size_t>(1, S.small_tmpl.size()) * sizeof(SmallParams));
        if (err == cudaSuccess) err = cudaMalloc(&S.d_cnt[dir], (kPersistHeadWords + nt) * sizeof(unsigned));
        if (err == cudaSuccess && nt)
            err = cudaMemcpy(S.d_tasks[dir], S.tasks[dir].data(), nt * sizeof(PersistTask), cudaMemcpyHostToDevice);
        if (err == cudaSuccess && ni)
            err = cudaMemcpy(S.d_items[dir], S.items[dir].data(), ni * sizeof(int2), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) {
            free_dev(S, dir);
            return mg_cuda_fail(err, "batch: persistent work list");
        }
    }
    if (!S.d_status) {
        err = cudaMalloc(&S.d_status, 2 * sizeof(unsigned));
        if (err == cudaSuccess) err = cudaMemset(S.d_status, 0, 2 * sizeof(unsigned));
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: status words");
    }
    return MGARD_OK;
}

// The level table and small-tail parameters for a set of pointers.
void persist_tables(Persist &S, int dir, void *const *d_data, char *ws)
{
    auto &lv = S.h_lv[dir];
    auto &sp = S.h_small[dir];
    lv.assign(S.nlevels, PersistLevel());
    sp = S.small_tmpl;
    for (size_t fi = 0; fi < S.f.size(); ++fi) {
        const PField &F = S.f[fi];
        char *base = ws + F.off;
        for (int j = 0; j < F.nd; ++j) {
            PersistLevel &L = lv[F.lv_base + j];
            const PlanLevelView &v = F.lv[j];
            L.X = (j == 0) ? d_data[fi] : (void *)(base + F.v_off[j - 1]);
            L.V = base + F.v_off[j];
            L.F = base + F.f_off[j];
            L.G = base + F.g_off[j];
            for (int d = 0; d < 3; ++d) {
                L.n[d] = (int)v.n[d];
                L.m[d] = (int)v.m[d];
                L.w[d] = v.w[d];
                L.k[d] = v.k[d];
                L.fac[d] = v.fac[d];
                L.co[d] = v.co[d];
            }
            L.first = (j == 0) ? 1 : 0;
        }
        if (F.small >= 0) sp[F.small].A = base + F.v_off[F.nd - 1];
    }
}

template <typename TX, typename TW>
cudaError_t persist_launch_t(int dir, const PersistParams &p, int grid, size_t smem, cudaStream_t st)
{
    return launch_persist<TX, TW>(dir == 0 ? MODE_DEC : MODE_REC, p, grid, smem, st);
}

cudaError_t persist_launch(const Persist &S, int dir, cudaStream_t st)
{
    PersistParams p;
    p.lv = S.d_lv[dir];
    p.tasks = S.d_tasks[dir];
    p.items = S.d_items[dir];
    p.small = S.d_small[dir];
    p.nitems = (int)S.items[dir].size();
    p.next = S.d_cnt[dir];
    p.zero = S.d_cnt[dir] + 1;
    p.done = S.d_cnt[dir] + kPersistHeadWords;
    p.status = S.d_status + dir;
    p.spin_limit = S.spin;
    p.stall = S.stall;
    p.prof = S.prof_on ? S.d_prof + dir * kPersistProfWords : nullptr;
    const size_t cnt = (kPersistHeadWords + S.tasks[dir].size()) * sizeof(unsigned);
    cudaError_t err = cudaMemsetAsync(S.d_cnt[dir], 0, cnt, st);
    if (err != cudaSuccess) return err;
    switch (S.dtype) {
    case MGARD_F32: return persist_launch_t<float, float>(dir, p, S.grid, S.smem, st);
    case MGARD_F64: return persist_launch_t<double, double>(dir, p, S.grid, S.smem, st);
    default: return persist_launch_t<float, double>(dir, p, S.grid, S.smem, st);
    }
}

mgard_status persist_run(mgard_batch *B, int dir, void *const *d_data, void *d_ws, cudaStream_t st)
{
    Persist &S = B->ps;
    const int n = (int)B->plans.size();
    const bool same = S.uploaded[dir] && S.ws[dir] == d_ws && (int)S.data[dir].size() == n &&
                      std::equal(S.data[dir].begin(), S.data[dir].end(), d_data);
    if (!same) {
        persist_tables(S, dir, d_data, static_cast<char *>(d_ws));
        // pageable copies: the host tables are copied out before the call returns
        cudaError_t err = cudaSuccess;
        if (S.nlevels)
            err = cudaMemcpyAsync(S.d_lv[dir], S.h_lv[dir].data(), S.h_lv[dir].size() * sizeof(PersistLevel),
                                  cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess && !S.h_small[dir].empty())
            err = cudaMemcpyAsync(S.d_small[dir], S.h_small[dir].data(), S.h_small[dir].size() * sizeof(SmallParams),
                                  cudaMemcpyHostToDevice, st);
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: level table upload");
        S.data[dir].assign(d_data, d_data + n);
        S.ws[dir] = d_ws;
        S.uploaded[dir] = true;
    }
    if (!S.exec[dir]) {
        // counter reset + launch, captured on an internal stream
        cudaStream_t origin = B->streams[0];
        cudaError_t err = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: begin capture");
        const cudaError_t lerr = persist_launch(S, dir, origin);
        cudaGraph_t graph = nullptr;
        err = cudaStreamEndCapture(origin, &graph);
        if (lerr != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return mg_cuda_fail(lerr, "batch: persistent kernel launch");
        }
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: end capture");
        err = cudaGraphInstantiate(&S.exec[dir], graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) {
            S.exec[dir] = nullptr;
            return mg_cuda_fail(err, "batch: graph instantiation");
        }
    }
    const cudaError_t err = cudaGraphLaunch(S.exec[dir], st);
    return err == cudaSuccess ? MGARD_OK : mg_cuda_fail(err, "batch: graph launch");
}

void persist_drop_graphs(Persist &S)
{
    for (int dir = 0; dir < 2; ++dir) {
        if (S.exec[dir]) cudaGraphExecDestroy(S.exec[dir]);
        S.exec[dir] = nullptr;
    }
}

}  // namespace

extern "C" {

mgard_status mgard_batch_destroy(mgard_batch *B)
{
    if (!B) return MGARD_OK;
    for (auto &g : B->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int dir = 0; dir < 2; ++dir) free_dev(B->ps, dir);
    cudaFree(B->ps.d_status);
    cudaFree(B->ps.d_prof);
    for (cudaEvent_t e : B->events) cudaEventDestroy(e);
    for (cudaStream_t s : B->streams) cudaStreamDestroy(s);
    delete B;
    return MGARD_OK;
}

mgard_status mgard_batch_create(int nfields, mgard_plan *const *plans, int nstreams, mgard_batch **out)
{
    if (!out) return MGARD_ERR_INVALID_ARG;
    *out = nullptr;
    if (nfields < 1 || !plans || nstreams < 1 || nstreams > 32) return MGARD_ERR_INVALID_ARG;
    for (int i = 0; i < nfields; ++i)
        if (!plans[i]) return MGARD_ERR_INVALID_ARG;
    mgard_batch *B = new (std::nothrow) mgard_batch();
    if (!B) return MGARD_ERR_INTERNAL;
    B->plans.assign(plans, plans + nfields);
    // workspace slices, and a largest-first assignment of fields to streams
    std::vector<int> order(nfields);
    std::vector<size_t> work(nfields);
    for (int i = 0; i < nfields; ++i) {
        order[i] = i;
        work[i] = mgard_workspace_bytes(plans[i]) + 1;
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    const int ns = std::min(nstreams, nfields);
    std::vector<size_t> load(ns, 0);
    B->stream_of.assign(nfields, 0);
    for (int i : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->stream_of[i] = s;
        load[s] += work[i];
    }
    B->offsets.resize(nfields);
    size_t off = 0;
    for (int i = 0; i < nfields; ++i) {
        B->offsets[i] = off;
        off += align_up(mgard_workspace_bytes(plans[i]));
    }
    B->graph_ws = off;
    cudaError_t err = cudaSuccess;
    for (int s = 0; s < ns && err == cudaSuccess; ++s) {
        cudaStream_t st;
        err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (err == cudaSuccess) B->streams.push_back(st);
    }
    for (int e = 0; e < ns + 1 && err == cudaSuccess; ++e) {
        cudaEvent_t ev;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err == cudaSuccess) B->events.push_back(ev);
    }
    if (err != cudaSuccess) {
        mgard_batch_destroy(B);
        return MGARD_ERR_CUDA;
    }
    Persist &S = B->ps;
    S.eligible = persist_analyse(B->plans, S);
    if (S.eligible) {
        const mgard_status st = persist_build(S);
        if (st != MGARD_OK) {
            mgard_batch_destroy(B);
            return st;
        }
        S.on = true;
    }
    B->ws_bytes = std::max(B->graph_ws, S.eligible ? S.ws_bytes : 0);
    *out = B;
    return MGARD_OK;
}

size_t mgard_batch_workspace_bytes(const mgard_batch *B) { return B ? B->ws_bytes : 0; }

static mgard_status batch_run(mgard_batch *B, int dir, void *const *d_data, void *d_ws, size_t ws_bytes,
                              void *stream)
{
    if (!B || !d_data) return mg_fail(MGARD_ERR_INVALID_ARG, "batch: NULL batch or data array");
    if (B->ws_bytes > 0 && (!d_ws || ws_bytes < B->ws_bytes))
        return mg_fail(MGARD_ERR_WORKSPACE, "batch: workspace missing or too small");
    if (reinterpret_cast<uintptr_t>(d_ws) % kSliceAlign != 0)
        return mg_fail(MGARD_ERR_WORKSPACE, "batch: workspace must be 256-byte aligned");
    const int n = (int)B->plans.size();
    for (int i = 0; i < n; ++i)
        if (!d_data[i]) return mg_fail(MGARD_ERR_INVALID_ARG, "batch: NULL field pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B->ps.on) return persist_run(B, dir, d_data, d_ws, st);
    Graph &G = B->graphs[dir];
    const bool same = G.exec && G.ws == d_ws && (int)G.data.size() == n &&
                      std::equal(G.data.begin(), G.data.end(), d_data);
    if (!same) {
        if (G.exec) {
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        // relaxed capture on the first internal stream: the launchers'
        // one-time function-attribute calls are allowed while capturing
        cudaStream_t origin = B->streams[0];
        cudaError_t err = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: begin capture");
        mgard_status status = MGARD_OK;
        const int ns = (int)B->streams.size();
        cudaEventRecord(B->events[0], origin);
        for (int s = 1; s < ns; ++s) cudaStreamWaitEvent(B->streams[s], B->events[0], 0);
        for (int i = 0; i < n && status == MGARD_OK; ++i) {
            char *ws = static_cast<char *>(d_ws) + B->offsets[i];
            const size_t wsb = mgard_workspace_bytes(B->plans[i]);
            cudaStream_t fs = B->streams[B->stream_of[i]];
            // per-field kernels only: a cooperative launch would hold every
            // SM and serialize the fields
            status = mg_transform(B->plans[i], dir, d_data[i], ws, wsb, fs, false);
        }
        for (int s = 1; s < ns; ++s) {
            cudaEventRecord(B->events[s], B->streams[s]);
            cudaStreamWaitEvent(origin, B->events[s], 0);
        }
        cudaGraph_t graph = nullptr;
        err = cudaStreamEndCapture(origin, &graph);
        if (status != MGARD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return status;
        }
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: end capture");
        err = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) {
            G.exec = nullptr;
            return mg_cuda_fail(err, "batch: graph instantiation");
        }
        G.data.assign(d_data, d_data + n);
        G.ws = d_ws;
    }
    const cudaError_t err = cudaGraphLaunch(G.exec, st);
    return err == cudaSuccess ? MGARD_OK : mg_cuda_fail(err, "batch: graph launch");
}

mgard_status mgard_batch_decompose(mgard_batch *B, void *const *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    return batch_run(B, 0, d_data, d_ws, ws_bytes, stream);
}

mgard_status mgard_batch_recompose(mgard_batch *B, void *const *d_data, void *d_ws, size_t ws_bytes, void *stream)
{
    return batch_run(B, 1, d_data, d_ws, ws_bytes, stream);
}

mgard_status mgard_batch_tune(mgard_batch *B, int param, int value)
{
    if (!B) return MGARD_ERR_INVALID_ARG;
    Persist &S = B->ps;
    switch (param) {
    case 0:  // 1: the persistent kernel, 0: the graph of per-field launches
        if (value != 0 && value != 1) return MGARD_ERR_INVALID_ARG;
        if (value == 1 && !S.eligible) return mg_fail(MGARD_ERR_INVALID_ARG, "batch: " + S.why);
        S.on = value == 1;
        return MGARD_OK;
    case 1:  // dependency polls before a wait gives up
        if (value < 1) return MGARD_ERR_INVALID_ARG;
        S.spin = value;
        persist_drop_graphs(S);
        return MGARD_OK;
    case 2:  // test hook: the first item waits for a count nothing reaches
        if (value != 0 && value != 1) return MGARD_ERR_INVALID_ARG;
        S.stall = value;
        persist_drop_graphs(S);
        return MGARD_OK;
    case 4:  // measurement: busy and waiting time per item kind
        if (value != 0 && value != 1) return MGARD_ERR_INVALID_ARG;
        if (value && !S.d_prof) {
            const size_t b = 2 * kPersistProfWords * sizeof(unsigned long long);
            cudaError_t err = cudaMalloc(&S.d_prof, b);
            if (err == cudaSuccess) err = cudaMemset(S.d_prof, 0, b);
            if (err != cudaSuccess) return mg_cuda_fail(err, "batch: profile counters");
        }
        S.prof_on = value == 1;
        persist_drop_graphs(S);
        return MGARD_OK;
    case 5:  // queue order (0: fields by size, 1: longest remaining path first)
        if (value != 0 && value != 1) return MGARD_ERR_INVALID_ARG;
        if (!S.eligible) return mg_fail(MGARD_ERR_INVALID_ARG, "batch: " + S.why);
        S.order = value;
        return persist_build(S);
    case 3:  // blocks per SM (0: as many as fit)
        if (value < 0 || value > 32) return MGARD_ERR_INVALID_ARG;
        if (!S.eligible) return mg_fail(MGARD_ERR_INVALID_ARG, "batch: " + S.why);
        S.bps_req = value;
        return persist_build(S);
    default: return MGARD_ERR_INVALID_ARG;
    }
}

long long mgard_batch_get(const mgard_batch *B, int param)
{
    if (!B) return -1;
    const Persist &S = B->ps;
    switch (param) {
    case 0: return S.on ? 1 : 0;
    case 1: return S.spin;
    case 2: return S.stall;
    case 3: return S.bps_req;
    case 4: return S.eligible ? 1 : 0;
    case 5: return S.grid;
    case 6: return S.occupancy;
    case 7: return (long long)S.items[0].size();
    case 8: return (long long)S.items[1].size();
    case 9: return (long long)(S.model_ns[0] / 1000.0);
    case 10: return (long long)(S.model_ns[1] / 1000.0);
    case 11: return (long long)S.smem;
    case 12: return S.order;
    default: return -1;
    }
}

mgard_status mgard_batch_profile_read(mgard_batch *B, int dir, double *busy_ms, double *wait_ms, long long *items)
{
    if (!B || dir < 0 || dir > 1 || !busy_ms || !wait_ms || !items) return MGARD_ERR_INVALID_ARG;
    Persist &S = B->ps;
    unsigned long long h[kPersistProfWords] = {};
    if (S.d_prof) {
        cudaError_t err = cudaDeviceSynchronize();
        if (err == cudaSuccess)
            err = cudaMemcpy(h, S.d_prof + dir * kPersistProfWords, sizeof(h), cudaMemcpyDeviceToHost);
        if (err == cudaSuccess) err = cudaMemset(S.d_prof + dir * kPersistProfWords, 0, sizeof(h));
        if (err != cudaSuccess) return mg_cuda_fail(err, "batch: profile read");
    }
    for (int k = 0; k < kPersistKinds; ++k) {
        busy_ms[k] = h[k] * 1e-6;
        wait_ms[k] = h[kPersistKinds + k] * 1e-6;
        items[k] = (long long)h[2 * kPersistKinds + k];
    }
    return MGARD_OK;
}

mgard_status mgard_batch_check(mgard_batch *B, void *stream)
{
    if (!B) return MGARD_ERR_INVALID_ARG;
    if (!B->ps.d_status) return MGARD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaStreamSynchronize(st);
    unsigned h[2] = {0, 0};
    if (err == cudaSuccess) err = cudaMemcpy(h, B->ps.d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemset(B->ps.d_status, 0, sizeof(h));
    if (err != cudaSuccess) return mg_cuda_fail(err, "batch: status read");
    if (h[0] | h[1]) return mg_fail(MGARD_ERR_TIMEOUT, "batch: a dependency wait of the persistent kernel ran out");
    return MGARD_OK;
}

}  // extern "C"
