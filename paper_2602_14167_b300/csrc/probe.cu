// FMA throughput probe (tcng_fma_peak): the FP32 / FP64 rate the SIMT kernels
// (the adjoint sweep, the expectation products) are measured against.
//
// Every thread runs eight independent FMA chains (enough to cover the pipe's
// latency) for a fixed number of iterations; grid = 8 CTAs of 256 threads per
// SM.  FLOPs = 2 x chains x iterations x threads; timed with CUDA events
// around one launch after a warm-up launch.  A measurement utility: it
// synchronises the device.
#include <cuda_runtime.h>

#include "capi_internal.hpp"

namespace tcng {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T* __restrict__ sink, int iters, T a, T b) {
    T x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == (T)12345.678) sink[0] = s;   // keeps the chains live; never true for these inputs
}

template <typename T>
tcng_status probe(double* tflops) {
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return fail(TCNG_ENOMEM, "probe buffer");
    const int blocks = num_sms() * 8;
    const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 11;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    fma_probe_kernel<T><<<blocks, kProbeThreads>>>(sink, iters / 4, a, b);
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<blocks, kProbeThreads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "FMA probe");
    const double flops = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return TCNG_OK;
}

}  // namespace
}  // namespace tcng

using namespace tcng;

extern "C" tcng_status tcng_fma_peak(int fp64, double* tflops) {
    if (!tflops) return fail(TCNG_EINVAL, "tflops is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    return fp64 ? probe<double>(tflops) : probe<float>(tflops);
}
