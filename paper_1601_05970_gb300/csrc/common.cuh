// Device-side state and deterministic reductions shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftg {

constexpr int kThreads = 256;

// Device material table: per phase K, G, sigma_0, H, n, eps_0, t_0, model
// (the fields of fftg_phase, the model id as a double).
constexpr int kMatStride = 8;
enum : int { MODEL_J2 = 0, MODEL_NLELASTIC = 1, MODEL_VISCO = 2 };

// Roundoff floor (relative to the norm of the projected field) below which a
// CG residual is treated as FFT roundoff; see the CG readings.
constexpr double kRoundoffRel = 1e-13;

// CG status values in CGState::done. CG_STAGNATED ends an inner (FP32)
// solve that has stopped improving: no new minimum of <r, r> for
// `stag_window` iterations, or a finite <p, q> <= 0 (rounding noise has
// overtaken the search direction). The iterate is kept and the FP64 Newton
// iteration refines it. CG_BREAKDOWN is a NaN or Inf.
enum : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3, CG_STAGNATED = 4 };

// State of one CG solve (one right-hand side), resident on the device so
// that the iteration needs no host round trip. The last block of each
// reducing kernel updates it.
struct CGState {
    double rr;       // <r, r> of the current residual
    double rr0;      // <r0, r0>
    double gs2;      // ||G sigma||^2 of the right-hand side before rounding
    double tol2;     // relative tolerance squared (set by the host)
    double floor2;   // absolute roundoff floor squared
    double stop2;    // max(tol2 * rr0, floor2)
    double pq;       // <p, q>
    double alpha;
    double beta;
    double omega;    // > 0: Richardson iteration with this fixed step (the
                     // basic scheme, Section 3.2) instead of CG; 0: CG
    double rr_min;   // smallest <r, r> so far
    int it_min;      // iteration of rr_min
    int stag_window; // > 0: stagnation test window (set by the host)
    int it;          // iterations done
    int max_it;      // cap (set by the host)
    int fixed_it;    // > 0: exactly this many iterations (set by the host)
    int done;        // CG_* status
    unsigned int ticket;  // last-block counter (always 0 between kernels)
    int pend;        // 1: x still lacks alpha p of the last update (the next
                     // P1 or the finishing kernel adds it)
};

// Scalars of one Newton iteration / one constitutive evaluation.
struct NewtonDev {
    double sig2;      // ||sigma||^2 (Frobenius, summed over voxels)
    double sum[6];    // sum of sigma over voxels, per component
    double de2;       // ||d eps||^2 of the last Newton update
    double extra[8];  // reductions of auxiliary kernels (tangent averages)
    unsigned int ticket;
    int nplastic;     // unused slot kept for alignment
};

// Transitions of a CGState, taken by thread 0 of the last block of a
// reducing kernel once the block totals are in.
//
// Start of a solve, after the right-hand side pass: rr = <r0, r0> in the
// inner precision, gs2 = ||G sigma||^2 before rounding to it.
__device__ __forceinline__ void cg_start(CGState* cg, double rr, double gs2) {
    cg->rr = rr;
    cg->rr0 = rr;
    cg->rr_min = rr;
    cg->it_min = 0;
    cg->gs2 = gs2;
    cg->it = 0;
    cg->beta = 0.0;
    cg->alpha = 0.0;
    const double stop2 = fmax(cg->tol2 * rr, cg->floor2);
    cg->stop2 = stop2;
    if (!isfinite(rr) || !isfinite(gs2)) {
        cg->done = CG_BREAKDOWN;
    } else if (gs2 <= cg->floor2 || rr == 0.0) {
        cg->done = CG_CONVERGED;
    } else if (cg->fixed_it <= 0 && rr <= stop2) {
        cg->done = CG_CONVERGED;
    } else {
        cg->done = CG_RUNNING;
    }
}

// After the matvec of an iteration: alpha = <r, r>/<p, q>, or the fixed
// Richardson step.
__device__ __forceinline__ void cg_after_dot(CGState* cg, double pq) {
    cg->pq = pq;
    cg->pend = 0;  // P1 of this iteration has added the previous step
    if (!isfinite(pq)) {
        cg->done = CG_BREAKDOWN;
    } else if (cg->omega > 0.0) {
        cg->alpha = cg->omega;  // Richardson: fixed step, <p, q> unused
    } else if (!(pq > 0.0)) {
        cg->done = cg->stag_window > 0 ? CG_STAGNATED : CG_BREAKDOWN;
    } else {
        cg->alpha = cg->rr / pq;
    }
}

// After r -= alpha q: rr = <r, r>; beta and the stopping tests. The step
// x += alpha p is left pending.
__device__ __forceinline__ void cg_after_update(CGState* cg, double rr) {
    const int it = cg->it + 1;
    cg->it = it;
    cg->pend = 1;
    cg->beta = cg->omega > 0.0 ? 0.0 : rr / cg->rr;  // Richardson: p = r
    cg->rr = rr;
    if (!isfinite(rr)) {
        cg->done = CG_BREAKDOWN;
    } else if (cg->fixed_it > 0) {
        if (it >= cg->fixed_it) cg->done = CG_CONVERGED;
    } else if (rr <= cg->stop2) {
        cg->done = CG_CONVERGED;
    } else if (it >= cg->max_it) {
        cg->done = CG_MAXIT;
    } else if (cg->stag_window > 0) {
        if (rr < cg->rr_min) {
            cg->rr_min = rr;
            cg->it_min = it;
        } else if (it - cg->it_min >= cg->stag_window) {
            cg->done = CG_STAGNATED;
        }
    }
}

// Frobenius product of symmetric tensors stored as 6 components
template <typename T>
__device__ __forceinline__ T frob(const T* a, const T* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + T(2) * (a[3] * b[3] + a[4] * b[4] + a[5] * b[5]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of kThreads threads (1D); result valid in every thread.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kThreads / 32];
    __shared__ double total;
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double s = (lane < kThreads / 32) ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) total = s;
    }
    __syncthreads();
    return total;
}

// Sum over a block of any size up to 1024 threads (1D), in a fixed order
// (lanes by shuffles, then the warps in index order); result in thread 0.
__device__ __forceinline__ double block_sum_any(double v) {
    __shared__ double red_any[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red_any[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) s += red_any[w];
    return s;
}

// <r, r> of the fused CG iteration from the block partials P5 wrote
// ([nf][nb], one per block): one block per field sums them in a fixed order
// and takes the CG state's update step (beta and the stopping tests).
static __global__ void __launch_bounds__(1024) k_cg_rr(const double* partials, int nb, CGState* cg) {
    const int f = blockIdx.x;
    if (cg[f].done) return;
    const double* in = partials + (size_t)f * nb;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += in[b];
    acc = block_sum_any(acc);
    if (threadIdx.x == 0) cg_after_update(cg + f, acc);
}

// Store this block's NV partial sums and report whether this block is the
// last one of `nblocks` to do so. Partials of the other blocks are then
// visible to it (fence before the ticket).
template <int NV>
__device__ __forceinline__ bool publish_partials(const double (&v)[NV], double* partials, int bid,
                                                 int nblocks, unsigned int* ticket) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)bid * NV + j] = v[j];
        __threadfence();
        unsigned int prev = atomicAdd(ticket, 1u);
        last = (prev == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    return last;
}

// In the last block: totals over all blocks in a fixed order (thread i takes
// blocks i, i + kThreads, ...; then a fixed tree), so the result does not
// depend on which block finished last. Resets the ticket.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* partials, int nblocks, unsigned int* ticket,
                                                double (&tot)[NV]) {
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += __ldcg(partials + (size_t)b * NV + j);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = block_sum(acc[j]);
    if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace fftg
