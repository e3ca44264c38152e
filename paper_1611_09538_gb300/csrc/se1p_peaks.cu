// FMA-loop microbenchmark: the FP32 and FP64 arithmetic peaks of the current
// device, measured with the same clocks and power state as the evaluation that
// is being reported.  The gridding, gathering and real-space kernels are bound
// by FP32 (mixed precision) or FP64 arithmetic, not by HBM bandwidth; their
// roofline fractions are taken against these rates.
#include <cuda_runtime.h>

#include "se1p_plan.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;  // independent FMA chains per thread (covers the pipe latency)

// Every thread runs kPeakChains dependent chains of `iters` FMAs each; the result is
// written only when it equals an impossible value, so the compiler keeps the work.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_loop(int iters, T a, T b, T *sink)
{
    T v[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kPeakChains; ++c) v[c] = v[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += v[c];
    if (s == (T)-12345.678) sink[blockIdx.x] = s;
}

template <typename T> se1p_status measure(int iters, double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return SE1P_ERR_CUDA;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_loop<T>, kPeakThreads, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        return SE1P_ERR_CUDA;
    }
    const int blocks = sms * per_sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return SE1P_ERR_CUDA;
    }
    // a = 1 - 2^-20 and b small keep the values finite and away from denormals
    const T a = (T)(1.0 - 1.0 / (1 << 20)), b = (T)1e-6;
    k_fma_loop<T><<<blocks, kPeakThreads>>>(iters / 8, a, b, nullptr);  // warm-up (clocks ramp)
    constexpr int kReps = 3;
    float best = 0.f;
    bool ok = cudaGetLastError() == cudaSuccess;
    for (int r = 0; ok && r < kReps; ++r) {
        cudaEventRecord(e0);
        k_fma_loop<T><<<blocks, kPeakThreads>>>(iters, a, b, nullptr);
        cudaEventRecord(e1);
        float ms = 0.f;
        ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || best <= 0.f) {
        cudaGetLastError();
        return SE1P_ERR_CUDA;
    }
    const double flops = 2.0 * (double)blocks * kPeakThreads * kPeakChains * (double)iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    return SE1P_OK;
}

}  // namespace

extern "C" se1p_status se1p_measure_fma_peak(int precision, double *tflops, int *sm_count)
{
    if (!tflops || (precision != SE1P_FP64 && precision != SE1P_MIXED)) return SE1P_ERR_INVALID_ARG;
    if (sm_count) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return SE1P_ERR_CUDA;
        }
    }
    // about 10 ms per timed launch on a GB300-class part in either precision
    return precision == SE1P_MIXED ? measure<float>(1 << 17, tflops) : measure<double>(1 << 12, tflops);
}
