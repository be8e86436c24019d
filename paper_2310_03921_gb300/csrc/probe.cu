// Throughput probes for the roofline denominators of ALU-bound kernels:
// FP32 and FP64 fused multiply-add rates of this GPU, measured with CUDA
// events over independent FMA chains (eight per thread, one CTA per SM
// slot), so that the issue rate, not latency, bounds them.
#include <string>

#include "gap_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T b, T c)
{
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = (T)(threadIdx.x + u);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = a[u] * b + c;
    }
    T s = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains live
}

template <typename T> gap_status probe(int iters, double *tflops)
{
    int dev = 0, sms = 0;
    GAP_TRY_CUDA(cudaGetDevice(&dev));
    GAP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    T *out = nullptr;
    GAP_TRY_CUDA(cudaMalloc(&out, sizeof(T) * blocks));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, 0);
        k_fma_chains<T><<<blocks, 256>>>(out, iters, (T)0.999999, (T)1e-6);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first run is a warm-up
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return gap_cuda_status(err, "k_fma_chains");
    *tflops = 2.0 * 8.0 * iters * 256.0 * blocks / (best * 1e-3) / 1e12;
    return GAP_OK;
}

}  // namespace

extern "C" gap_status gap_test_fma_peak(int fp64, double *tflops)
{
    if (!tflops) {
        gap_set_error("tflops is NULL");
        return GAP_EINVAL;
    }
    return fp64 ? probe<double>(1 << 10, tflops) : probe<float>(1 << 14, tflops);
}
