// probe.cu -- measurement support: the FP64 fused multiply-add rate of the
// current GPU, the denominator of the FP64 compute roofline (the FP32 path
// is bound by HBM bandwidth, the FP64 one may be bound by the FP64 units).
#include <cuda_runtime.h>

#include <string>

#include "mgard.h"

mgard_status mg_fail(mgard_status st, const std::string &msg);
mgard_status mg_cuda_fail(cudaError_t err, const char *what);

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// Every thread runs kChains independent recurrences x = x * a + b for
// `iters` steps: 2 flops per step and chain.  The result is stored only if
// it is a value the recurrences cannot produce, so the work is kept.
__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(int iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" mgard_status mgard_probe_fp64_peak(double *tflops, void *stream)
{
    if (!tflops) return mg_fail(MGARD_ERR_INVALID_ARG, "probe_fp64_peak: tflops is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, bps = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_dfma_probe, kProbeThreads, 0);
    if (err != cudaSuccess) return mg_cuda_fail(err, "probe_fp64_peak: device query");
    const int grid = sms * (bps > 0 ? bps : 1);
    const int iters = 1 << 14;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    // a = 1 - 2^-30, b = 2^-10: the chains stay finite and non-trivial
    const double a = 1.0 - 0x1p-30, b = 0x1p-10;
    float ms = 0.f;
    if (err == cudaSuccess) {
        k_dfma_probe<<<grid, kProbeThreads, 0, st>>>(iters / 8, a, b, nullptr);  // warm-up
        err = cudaEventRecord(e0, st);
    }
    if (err == cudaSuccess) {
        k_dfma_probe<<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return mg_cuda_fail(err, "probe_fp64_peak");
    const double flops = 2.0 * kChains * (double)iters * grid * kProbeThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return MGARD_OK;
}
