// batch.cu -- batches of independent fields replayed as one CUDA graph.
//
// Every field has its own plan and its own slice of the batch workspace, so
// fields are independent.  On the first call for a set of pointers the
// batch captures, on `stream`, a fork over `streams` internal streams (fields
// assigned largest first to the least loaded stream), each field's level
// kernels on its stream, and the join back; later calls with the same
// pointers replay the instantiated graph with a single launch.
#include <algorithm>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mgard.h"

mgard_status mg_fail(mgard_status st, const std::string &msg);
mgard_status mg_cuda_fail(cudaError_t err, const char *what);
mgard_status mg_transform(const mgard_plan *P, int dir, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st,
                          bool allow_coop);

namespace {

constexpr size_t kSliceAlign = 256;

struct Graph {
    std::vector<void *> data;
    void *ws = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct mgard_batch {
    std::vector<mgard_plan *> plans;
    std::vector<size_t> offsets;     // workspace slice of each field
    std::vector<int> stream_of;      // internal stream of each field
    size_t ws_bytes = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // fork event + one join event per stream
    Graph graphs[2];                  // decompose, recompose
};

extern "C" {

mgard_status mgard_batch_destroy(mgard_batch *B)
{
    if (!B) return MGARD_OK;
    for (auto &g : B->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
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
        off += (mgard_workspace_bytes(plans[i]) + kSliceAlign - 1) / kSliceAlign * kSliceAlign;
    }
    B->ws_bytes = off;
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

}  // extern "C"
