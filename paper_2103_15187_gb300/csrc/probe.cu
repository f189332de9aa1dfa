// Measurement helper: the device's double-precision fused multiply-add
// throughput, the denominator of the FP64 step's arithmetic roofline (the
// FP64 step is bound by the FP64 pipe, not by memory).  Not part of the
// method; nothing on the step's path calls it.
#include "../../include/fsei.h"
#include "common.cuh"

namespace {

// written only if a chain ever produced the impossible value below, which
// keeps the compiler from dropping the arithmetic
__device__ double g_fma_sink;

constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kThreads = 256;

// Each thread runs kChains independent chains a <- a * b + c for iters
// iterations: kChains * iters DFMA instructions per thread, enough
// independent work per warp to keep the FP64 pipe busy.
__global__ void __launch_bounds__(kThreads) k_fp64_fma(int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.2345e300) g_fma_sink = s;
}

}  // namespace

extern "C" fsei_status fsei_fp64_fma_rate(void *cuda_stream, double *ginst_per_s) {
    if (!ginst_per_s) return FSEI_E_ARG;
    *ginst_per_s = 0.0;
    cudaGetLastError();
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSEI_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FSEI_E_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, kThreads, 0) !=
            cudaSuccess || per_sm < 1)
        return FSEI_E_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * per_sm;
    const int iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FSEI_E_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FSEI_E_CUDA;
    }
    // |b| < 1 keeps the chains bounded (they converge to c / (1 - b))
    k_fp64_fma<<<blocks, kThreads, 0, st>>>(iters / 8, 0.999999, 1e-6);
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, kThreads, 0, st>>>(iters, 0.999999, 1e-6);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || !(best > 0.f)) return FSEI_E_CUDA;
    const double inst = (double)blocks * kThreads * kChains * iters;
    *ginst_per_s = inst / (best * 1e-3) / 1e9;
    return FSEI_OK;
}
