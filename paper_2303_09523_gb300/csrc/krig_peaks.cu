// krig_peaks.cu -- arithmetic peak microbenchmarks (FP32 and FP64 fused
// multiply-add issue rates) used as roofline denominators for the kernels
// whose bound is the ALU rather than HBM.  Each thread runs 8 independent FMA
// chains so the pipe, not latency, is the limit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "krig_internal.h"

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (T)1234.5) out[blockIdx.x] = s;  // keeps the chains live
}

template <typename T>
static krig_status run_peak(double* gflops)
{
    int sms = krig_device_sm_count();
    if (sms <= 0) return KRIG_ECUDA;
    T* out = nullptr;
    const int blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 64 : 4096;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return KRIG_ECUDA;
    k_fma_peak<T><<<blocks, 256>>>(out, iters / 8, (T)0.999, (T)0.001);  // warm-up
    cudaEventRecord(a);
    k_fma_peak<T><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess || ms <= 0.f) return KRIG_ECUDA;
    const double fmas = (double)blocks * 256.0 * iters * 16.0 * 8.0;
    *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
    return KRIG_OK;
}

extern "C" krig_status krig_measure_fma_peak(int32_t fp64, double* gflops_out)
{
    if (!gflops_out) return KRIG_EINVAL;
    return fp64 ? run_peak<double>(gflops_out) : run_peak<float>(gflops_out);
}
