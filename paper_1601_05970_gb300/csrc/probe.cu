// Arithmetic-throughput probe: the device's fused multiply-add rate in FP64
// or FP32, measured with CUDA events over one launch that keeps every SM
// busy with independent FMA chains. It gives the roofline denominator of
// the ALU-bound passes (the plain FP64 path); it is not part of the method.
#include <cuda_runtime.h>

#include "../../include/fftg.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// The chains stay positive, so no thread's sum is -1 and nothing is stored:
// the conditional store only keeps the chains live.
__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1)) g_probe_sink = (double)s;
}

template <typename T>
int probe(int iters, cudaStream_t s, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FFTG_ECUDA;
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FFTG_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FFTG_ECUDA;
    }
    // a = 1 - 2^-20, b = 2^-20: every chain stays bounded, so the rate does
    // not depend on denormals or infinities
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(iters / 8, a, b);  // warm-up
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(iters, a, b);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return FFTG_ECUDA;
    const double flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return FFTG_OK;
}

}  // namespace

extern "C" int fftg_probe_fma_rate(int precision, int iters, void* stream, double* tflops) {
    if (!tflops || iters < 8 || (precision != FFTG_FP64 && precision != FFTG_MIXED)) return FFTG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == FFTG_FP64 ? probe<double>(iters, s, tflops) : probe<float>(iters, s, tflops);
}
