// Throughput of the arithmetic pipes the solver's kernels run on, measured on the
// device they run on: the FP32 FMA pipe, the FP64 pipe and the MUFU reciprocal square
// root.  Each kernel keeps every SM busy with independent dependency chains (8 per
// thread, 16 warps per SM scheduler) and is timed with CUDA events over a loop long
// enough for the clocks to settle; the operation counts are exact.  A diagnostic for
// the roofline of the solver's row kernels, not part of the solve.
#include <cuda_runtime.h>

#include "sf.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(512) k_peak_ffma(int iters, float a, float b, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345f) sink[0] = s;   // keeps the chains alive; never true for these inputs
}

__global__ void __launch_bounds__(512) k_peak_dfma(int iters, double a, double b, double *sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345) sink[0] = s;
}

__global__ void __launch_bounds__(512) k_peak_rsqrt(int iters, float *sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345f) sink[0] = s;
}

// ms of one launch of `go` on every SM, best of 3 after a warm-up launch
template <typename F>
int time_it(F go, cudaStream_t st, float *best)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SF_ECUDA;
    }
    int rc = SF_OK;
    *best = 1e30f;
    for (int r = 0; r < 4 && rc == SF_OK; ++r) {
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = SF_ECUDA;
        go();
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            rc = SF_ECUDA;
        float ms = 0.f;
        if (rc == SF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SF_ECUDA;
        if (rc == SF_OK && r > 0 && ms < *best) *best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int sf_alu_peaks(double seconds, double *out, void *stream)
{
    if (!out || !(seconds > 0.0) || seconds > 60.0) return SF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    void *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return SF_ENOMEM;
    const int blocks = sms * 4, threads = 512;
    const double lanes = (double)blocks * threads * kChains;
    int rc = SF_OK;
    // a short probe sizes each loop to about seconds / 3 per timed launch
    auto sized = [&](auto launch, double ops_per_iter, double *rate) {
        int it = 1 << 14;
        float ms = 0.f;
        if ((rc = time_it([&] { launch(it); }, st, &ms)) != SF_OK) return;
        const double scale = (seconds / 3.0 * 1e3) / (double)(ms > 1e-3f ? ms : 1e-3f);
        it = (int)(it * (scale < 1.0 ? 1.0 : scale > 4096.0 ? 4096.0 : scale));
        if ((rc = time_it([&] { launch(it); }, st, &ms)) != SF_OK) return;
        *rate = lanes * (double)it * ops_per_iter / ((double)ms * 1e-3);
    };
    sized([&](int it) { k_peak_ffma<<<blocks, threads, 0, st>>>(it, 0.999f, 1e-3f, (float *)sink); }, 2.0, &out[0]);
    if (rc == SF_OK)
        sized([&](int it) { k_peak_dfma<<<blocks, threads, 0, st>>>(it, 0.999, 1e-3, (double *)sink); }, 2.0, &out[1]);
    if (rc == SF_OK)
        sized([&](int it) { k_peak_rsqrt<<<blocks, threads, 0, st>>>(it, (float *)sink); }, 1.0, &out[2]);
    cudaFree(sink);
    return rc;
}
