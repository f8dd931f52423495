// fftg_constitutive_noalloc: the J2 stress update with homogenisation for
// callers that cannot allocate device memory.
//
// Who needs it: a host program that has already reserved all of its device
// memory (a finite-element code running its own pool allocator, say, that
// evaluates the material law at its Gauss points from inside its assembly
// loop) cannot let a library call cudaMalloc: the allocation either fails
// because the pool holds the memory, or stalls every stream of the device
// while it runs. This entry point needs no handle and no workspace. The
// caller passes all inputs and outputs; the only other memory it touches
// is a fixed array compiled into this file.
//
// That array holds the per-block partial sums of the stress reduction, the
// finishing ticket, the material table and a flag for phase ids out of
// range. It is a static __device__ array, so every GPU that loads the
// library holds it until the process exits; its size is fixed below.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/fftg.h"
#include "materials.h"
#include "pointwise.cuh"

namespace {

using fftg::ConstArgs;
using fftg::NewtonDev;

constexpr int kMaxPhases = 256;
constexpr int kPartialBlocks = fftg::kMaxPointwiseBlocks;  // grid cap of the kernel

// Layout of the array: [partials: kPartialBlocks x 7 doubles]
// [material table: kMaxPhases x kMatStride doubles] [NewtonDev: sums and ticket]
// [flag: int, non-zero when a phase id is >= nphase].
constexpr size_t kOffPartials = 0;
constexpr size_t kOffMats = kOffPartials + (size_t)kPartialBlocks * 7 * sizeof(double);
constexpr size_t kOffNd = kOffMats + (size_t)kMaxPhases * fftg::kMatStride * sizeof(double);
constexpr size_t kOffFlag = kOffNd + ((sizeof(NewtonDev) + 15) / 16) * 16;
constexpr size_t kScratchBytes = ((kOffFlag + sizeof(int) + 255) / 256) * 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Sets *flag when any of the V phase ids is >= nphase. Phase ids are bytes,
// so the material table of kMaxPhases rows covers every id the stress
// kernel can read; rows at or past nphase hold NaN, and the call reports
// FFTG_EINVAL.
__global__ void k_phase_check(const uint8_t* __restrict__ phase, long long V, int nphase, int* flag) {
    int bad = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x)
        bad |= phase[v] >= nphase;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (in host code the symbol itself is only a host-side handle).
cudaError_t scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int fftg_constitutive_noalloc(int N, const double E[6], const double* eps_dev,
                                         const double* eps_p_dev, const double* epbar_dev,
                                         const uint8_t* phase_dev, int nphase, const fftg_phase* mats,
                                         int tangent_precision, void* tangent_dev, double* sigma_dev,
                                         double* eps_p_new_dev, double* epbar_new_dev,
                                         double sigma_mean[6], void* stream) {
    if (N < 1 || N > 243 || nphase < 1 || nphase > kMaxPhases) return FFTG_EINVAL;
    if (!E || !eps_dev || !eps_p_dev || !epbar_dev || !phase_dev || !mats || !sigma_mean) return FFTG_EINVAL;
    if (tangent_dev && tangent_precision != FFTG_FP64 && tangent_precision != FFTG_MIXED) return FFTG_EINVAL;
    for (int i = 0; i < nphase; ++i)
        if (!fftg::phase_valid(mats[i], false)) return FFTG_EINVAL;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return FFTG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char* b = (char*)base;
    double* partials = (double*)(b + kOffPartials);
    double* dmats = (double*)(b + kOffMats);
    NewtonDev* nd = (NewtonDev*)(b + kOffNd);
    int* flag = (int*)(b + kOffFlag);
    // the whole table is written on every call: the caller's phases, then
    // NaN rows, so that no row keeps an earlier call's materials
    double m[kMaxPhases * fftg::kMatStride];
    for (int i = 0; i < kMaxPhases * fftg::kMatStride; ++i) m[i] = NAN;
    for (int i = 0; i < nphase; ++i) fftg::pack_phase(mats[i], m + fftg::kMatStride * i);
    // the ticket and the flag must start at zero; the rest is overwritten
    if (cudaMemsetAsync(nd, 0, kOffFlag + sizeof(int) - kOffNd, s) != cudaSuccess) return FFTG_ECUDA;
    if (cudaMemcpyAsync(dmats, m, sizeof(m), cudaMemcpyHostToDevice, s) != cudaSuccess) return FFTG_ECUDA;
    ConstArgs a{};
    a.V = (long long)N * N * N;
    a.cs = a.V;  // caller fields are [6][N^3], unpadded
    for (int c = 0; c < 6; ++c) a.E[c] = E[c];
    a.eps = eps_dev;
    a.eps_p = eps_p_dev;
    a.epbar = epbar_dev;
    a.phase = phase_dev;
    a.mats = dmats;
    a.sigma = sigma_dev;
    a.eps_p_new = eps_p_new_dev;
    a.epbar_new = epbar_new_dev;
    a.tangent = tangent_dev;
    a.partials = partials;
    a.nd = nd;
    a.cg = nullptr;
    a.tie = 1e-12;
    a.dt = 1.0;  // unused: no rate-dependent phases here
    const int nb = fftg::pointwise_blocks(a.V);
    k_phase_check<<<nb, fftg::kThreads, 0, s>>>(phase_dev, a.V, nphase, flag);
    if (tangent_dev && tangent_precision == FFTG_FP64)
        fftg::k_constitutive<double><<<nb, fftg::kThreads, 0, s>>>(a);
    else
        fftg::k_constitutive<float><<<nb, fftg::kThreads, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FFTG_ECUDA;
    NewtonDev out;
    int bad = 0;
    if (cudaMemcpyAsync(&out, nd, sizeof(NewtonDev), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FFTG_ECUDA;
    if (bad) return FFTG_EINVAL;
    for (int c = 0; c < 6; ++c) sigma_mean[c] = out.sum[c] / (double)a.V;
    return FFTG_OK;
}
