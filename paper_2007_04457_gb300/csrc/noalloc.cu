// noalloc.cu -- decomposition that allocates no device memory.
//
// The regular entry points take a caller-allocated workspace and a plan that
// owns small device tables (allocated once, by mgard_plan_create).  Some
// callers cannot allocate device memory at the point where they need the
// transform: a process whose device memory is already held by its own pool
// allocator, or a loop that must not call cudaMalloc/cudaFree because those
// calls synchronize the whole device and stall every other stream.
// mgard_decompose_noalloc serves them: the tables and the workspace live in
// one file-scope device array of fixed size, created with the module, so no
// call allocates or frees device memory.
#include <cuda_runtime.h>

#include <string>

#include "mgard.h"

struct mgard_plan;
mgard_status mg_fail(mgard_status st, const std::string &msg);
mgard_status mg_cuda_fail(cudaError_t err, const char *what);
mgard_status mg_plan_in_place(int ndim, const int64_t *dims, int nlevels, mgard_dtype dtype, void *dev,
                              size_t dev_bytes, cudaStream_t stream, mgard_plan **out, size_t *used);
mgard_status mg_decompose_with(const mgard_plan *P, void *d_data, void *d_ws, size_t ws_bytes, cudaStream_t st);

namespace {

constexpr size_t kScratchBytes = MGARD_NOALLOC_SCRATCH_BYTES;

// The scratch: one copy per device, made when this module is loaded on it.
// Every call writes the tables and workspace regions it reads, so nothing
// here has to start at zero.
static __device__ __align__(256) unsigned char scratch[kScratchBytes];

}  // namespace

extern "C" mgard_status mgard_decompose_noalloc(int ndim, const int64_t *dims, int nlevels, mgard_dtype dtype,
                                                void *d_data, void *stream)
{
    if (!d_data) return mg_fail(MGARD_ERR_INVALID_ARG, "mgard_decompose_noalloc: d_data is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the tables are copied from host vectors that this call frees on return
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(st, &cap);
    if (err != cudaSuccess) return mg_cuda_fail(err, "mgard_decompose_noalloc: cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return mg_fail(MGARD_ERR_INVALID_ARG, "mgard_decompose_noalloc: the stream is being captured; this call cannot be");
    // the current device's copy of the scratch (host code only sees a
    // stand-in for the symbol; the lookup is cheap, so it is not cached)
    void *base = nullptr;
    err = cudaGetSymbolAddress(&base, scratch);
    if (err != cudaSuccess) return mg_cuda_fail(err, "mgard_decompose_noalloc: cudaGetSymbolAddress");
    mgard_plan *P = nullptr;
    size_t used = 0;
    mgard_status s = mg_plan_in_place(ndim, dims, nlevels, dtype, base, kScratchBytes, st, &P, &used);
    if (s != MGARD_OK) return s;
    s = mg_decompose_with(P, d_data, static_cast<unsigned char *>(base) + used, kScratchBytes - used, st);
    // the launches hold copies of what they need; the tables stay in the scratch
    const mgard_status sd = mgard_plan_destroy(P);
    return s != MGARD_OK ? s : sd;
}
