// mhd_peak.cu -- measured FP32 / FP64 fused multiply-add throughput of the
// device, the denominator of the arithmetic side of the roofline that the
// benchmark reports beside the HBM side.  Not part of the method: a
// measurement helper, timed with CUDA events on its own stream at whatever
// clocks the device runs (no clock or power setting is touched).
#include <cuda_runtime.h>
#include "mhd.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T* sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = x[c] * a + b;   // one FMA each
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == T(-1234.5)) *sink = s;   // keeps the chains live; never true for these inputs
}

template <class T>
mhd_status run(int iters, int reps, double* tflops)
{
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MHD_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MHD_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_chains<T>, kThreads, 0) != cudaSuccess || per < 1)
        per = 1;
    const int grid = nsm * per;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MHD_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a = 1 - 2^-20 keeps |x| bounded and away from denormals
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1e-6);
    k_fma_chains<T><<<grid, kThreads, 0, st>>>(iters, a, b, nullptr);   // warm-up
    float best = 1e30f;
    mhd_status s = MHD_OK;
    for (int r = 0; r < reps && s == MHD_OK; r++) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<grid, kThreads, 0, st>>>(iters, a, b, nullptr);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = MHD_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess) s = MHD_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (s != MHD_OK) return s;
    const double fmas = (double)grid * kThreads * (double)iters * 16.0 * kChains;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return MHD_OK;
}

}  // namespace

extern "C" mhd_status mhd_fma_peak(int precision, int reps, double* tflops)
{
    if (!tflops || reps < 1 || reps > 1000) return MHD_EINVAL;
    if (precision == MHD_FP32) return run<float>(4096, reps, tflops);
    if (precision == MHD_FP64) return run<double>(64, reps, tflops);
    return MHD_EINVAL;
}
