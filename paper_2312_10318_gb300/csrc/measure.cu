// Measured FP64 arithmetic ceiling of the device: the throughput of a plain
// chain of fused multiply-adds in double precision, against which the
// FP64-storage step (bound by the FP64 pipe on GB300, not by HBM) is reported.
#include <cuda_runtime.h>

#include "trtrlb.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

// Target of a store that keeps the chains live (never taken in practice).
__device__ double g_fma_sink;

__global__ void __launch_bounds__(kThreads) k_fp64_fma(long long iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-9 * (threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.0) g_fma_sink = s;   // the chains converge to 8 * 2^-10: never true
}

}  // namespace

extern "C" int trtrlb_fp64_fma_rate(void* stream, double seconds, double* tflops) {
    if (!tflops || !(seconds > 0.0)) return TRTRLB_EINVAL;
    int dev = 0, sms = 0, occ = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fp64_fma, kThreads, 0);
    if (e != cudaSuccess || occ < 1) return TRTRLB_ECUDA;
    const int grid = sms * occ;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // a = 1 - 2^-20, b = 2^-30: every chain stays finite and away from zero
    const double a = 1.0 - 1.0 / 1048576.0, b = 1.0 / 1073741824.0;
    long long iters = 1024;
    float ms = 0.f;
    // grow the launch until it lasts about `seconds` (at least 10 ms)
    for (int round = 0; round < 16 && e == cudaSuccess; ++round) {
        e = cudaEventRecord(e0, st);
        k_fp64_fma<<<grid, kThreads, 0, st>>>(iters, a, b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double target = seconds * 1e3 < 10.0 ? 10.0 : seconds * 1e3;
        if (ms >= 0.5 * target) break;
        const double grow = ms > 0.f ? target / ms : 64.0;
        iters = (long long)(iters * (grow > 64.0 ? 64.0 : grow)) + 1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return TRTRLB_ECUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)grid * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return TRTRLB_OK;
}
