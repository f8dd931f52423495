// Finite-strain driver: the Newton-CG scheme of Algorithm 1 with the
// deformation gradient in place of the strain (the extension Section 6
// names), one cell per handle. The grid passes are those of fs_passes.cuh;
// the pointwise kernels here evaluate St. Venant-Kirchhoff's stress, update
// the CG vectors, apply the Newton correction and form the macroscopic
// tangent's floors and averages. As in the small-strain
// driver, every number is computed on the device and the host reads a few
// scalars per Newton iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fftg_fs.h"
#include "fs_passes.cuh"
#include "host_common.h"

namespace fftg {
#define FFTG_FS_EXTERN_N(n) extern template cudaError_t run_fs_pass_n<n>(FsPassKind, const FsArgs&, cudaStream_t);
FFTG_FS_EXTERN_N(3)
FFTG_FS_EXTERN_N(5)
FFTG_FS_EXTERN_N(9)
FFTG_FS_EXTERN_N(15)
FFTG_FS_EXTERN_N(25)
FFTG_FS_EXTERN_N(27)
FFTG_FS_EXTERN_N(45)
FFTG_FS_EXTERN_N(75)
FFTG_FS_EXTERN_N(81)
FFTG_FS_EXTERN_N(125)
FFTG_FS_EXTERN_N(135)
FFTG_FS_EXTERN_N(225)
FFTG_FS_EXTERN_N(243)
#undef FFTG_FS_EXTERN_N

#define FFTG_FS_GRIDS(X) X(3) X(5) X(9) X(15) X(25) X(27) X(45) X(75) X(81) X(125) X(135) X(225) X(243)

cudaError_t run_fs_pass(int N, FsPassKind kind, const FsArgs& a, cudaStream_t s) {
    switch (N) {
#define FFTG_CASE(n) case n: return run_fs_pass_n<n>(kind, a, s);
        FFTG_FS_GRIDS(FFTG_CASE)
#undef FFTG_CASE
        default: return cudaErrorInvalidValue;
    }
}

int fs_row_blocks(int N, bool fp64) {
    switch (N) {
#define FFTG_CASE(n) case n: return fp64 ? FsCfg<n, double>::row_blocks : FsCfg<n, float>::row_blocks;
        FFTG_FS_GRIDS(FFTG_CASE)
#undef FFTG_CASE
        default: return 0;
    }
}

// ------------------------------------------------------------ pointwise
constexpr int kFsPointBlocks = 4096;

inline int fs_point_blocks(long long V) {
    const long long b = (V + kThreads - 1) / kThreads;
    return (int)(b < kFsPointBlocks ? b : kFsPointBlocks);
}

// Grid of the vectorised CG update: one thread per 16-byte vector of a
// component, capped (depends only on the grid size).
inline int fs_vector_blocks(long long cs, int elem_bytes) {
    const long long b = (cs / (16 / elem_bytes) + kThreads - 1) / kThreads;
    return (int)(b < kFsPointBlocks ? b : kFsPointBlocks);
}

// Scalars of one constitutive evaluation / Newton update.
struct FsDev {
    double p2;       // ||P||^2 (Frobenius, summed over voxels)
    double sum[9];   // sum of P over voxels
    double de2;      // ||dF*||^2 of the last Newton update
    unsigned int ticket;
    int pad;
};

struct FsPointArgs {
    long long V, cs;
    const double* Fbar;     // [9] on the device
    const double* Fs;       // F* [9][cs]
    double* P;              // [9][cs] or null
    void* hgrad;            // H = F - I [9][cs] in the inner precision, or null
    const uint8_t* phase;
    const double* lame;
    FsDev* dev;
    CGState* cg;            // constitutive: floor2 is set when not null
    double* partials;
    void* x;
    void* r;
    const void* p;
    const void* q;
    double* Fw;             // Newton update: F* += x
    int unit;               // tangent kernels: the perturbed component 3k + l
};

// P = F S with E = (H + H^T + H^T H)/2 (the Green-Lagrange strain written
// with H = F - I, which keeps small strains free of cancellation) and
// S = lambda tr(E) I + 2 mu E.
__device__ __forceinline__ void svk_stress(const double (&h)[9], double lam, double mu, double (&P)[9]) {
    double E[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double hh = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) hh += h[3 * k + i] * h[3 * k + j];
            E[3 * i + j] = 0.5 * (h[3 * i + j] + h[3 * j + i] + hh);
        }
    const double le = lam * (E[0] + E[4] + E[8]);
    double S[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) S[c] = 2.0 * mu * E[c] + ((c % 4 == 0) ? le : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double t = S[3 * i + j];  // (I + H) S
#pragma unroll
            for (int k = 0; k < 3; ++k) t += h[3 * i + k] * S[3 * k + j];
            P[3 * i + j] = t;
        }
}

// P(Fbar + F*) per voxel; H in the inner precision for the tangent; the
// totals ||P||^2 and sum P (fixed-order reduction); the CG roundoff floor.
template <typename TT>
__global__ void __launch_bounds__(kThreads) k_fs_constitutive(FsPointArgs a) {
    const long long V = a.V, cs = a.cs;
    double hb[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) hb[c] = a.Fbar[c] - ((c % 4 == 0) ? 1.0 : 0.0);
    double acc[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) acc[j] = 0.0;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        double h[9], P[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) h[c] = hb[c] + a.Fs[c * cs + v];
        const double* m = a.lame + 2 * a.phase[v];
        svk_stress(h, m[0], m[1], P);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            if (a.P) a.P[c * cs + v] = P[c];
            if (a.hgrad) ((TT*)a.hgrad)[c * cs + v] = (TT)h[c];
            acc[0] += P[c] * P[c];
            acc[1 + c] += P[c];
        }
    }
    double part[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) part[j] = block_sum(acc[j]);
    if (!publish_partials<10>(part, a.partials, blockIdx.x, gridDim.x, &a.dev->ticket)) return;
    double tot[10];
    reduce_partials<10>(a.partials, gridDim.x, &a.dev->ticket, tot);
    if (threadIdx.x != 0) return;
    a.dev->p2 = tot[0];
#pragma unroll
    for (int c = 0; c < 9; ++c) a.dev->sum[c] = tot[1 + c];
    if (a.cg) a.cg->floor2 = kRoundoffRel * kRoundoffRel * tot[0];
}

// r -= alpha q; <r, r>; beta and the stopping tests (x += alpha p deferred
// to the next P1 or to k_fs_cg_finish). 16-byte vectors over the padded
// components, all loads of an item before its stores; lanes in the padding
// are updated too (harmless) but left out of <r, r>.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fs_cg_update(FsPointArgs a) {
    CGState* cg = a.cg;
    if (cg->done) return;
    constexpr int VW = 16 / (int)sizeof(T);
    using VT = typename Vec16<T>::type;
    const long long V = a.V, nv = a.cs / VW;
    const T alpha = (T)cg->alpha;
    VT* r = (VT*)a.r;
    const VT* q = (const VT*)a.q;
    T acc = T(0);
    for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < nv;
         j += (long long)gridDim.x * kThreads) {
        VT rv[9], qv[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            rv[c] = r[c * nv + j];
            qv[c] = q[c * nv + j];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            T* re = reinterpret_cast<T*>(&rv[c]);
            const T* qe = reinterpret_cast<const T*>(&qv[c]);
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                re[e] -= alpha * qe[e];
                if (j * VW + e < V) acc += re[e] * re[e];
            }
            r[c * nv + j] = rv[c];
        }
    }
    double part[1] = {block_sum((double)acc)};
    if (!publish_partials<1>(part, a.partials, blockIdx.x, gridDim.x, &cg->ticket)) return;
    double tot[1];
    reduce_partials<1>(a.partials, gridDim.x, &cg->ticket, tot);
    if (threadIdx.x == 0) cg_after_update(cg, tot[0]);
}

// x += alpha p where the last update left the step pending.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fs_cg_finish(FsPointArgs a) {
    if (!a.cg->pend) return;
    const long long V = a.V, cs = a.cs;
    const T alpha = (T)a.cg->alpha;
    T* x = (T*)a.x;
    const T* p = (const T*)a.p;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
#pragma unroll
        for (int c = 0; c < 9; ++c) x[c * cs + v] += alpha * p[c * cs + v];
    }
}

// F* += x (Algorithm 1's update); dev->de2 = ||x||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fs_newton_update(FsPointArgs a) {
    const long long V = a.V, cs = a.cs;
    const T* x = (const T*)a.x;
    double acc = 0.0;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const double d = (double)x[c * cs + v];
            a.Fw[c * cs + v] += d;
            acc += d * d;
        }
    }
    double part[1] = {block_sum(acc)};
    if (!publish_partials<1>(part, a.partials, blockIdx.x, gridDim.x, &a.dev->ticket)) return;
    double tot[1];
    reduce_partials<1>(a.partials, gridDim.x, &a.dev->ticket, tot);
    if (threadIdx.x == 0) a.dev->de2 = tot[0];
}

// Macroscopic tangent, column `unit`: ||K : E_unit||^2 summed over voxels
// gives the CG roundoff floor of the right-hand side -G (K : E_unit).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fs_tangent_floor(FsPointArgs a) {
    const long long V = a.V, cs = a.cs;
    const T* hg = (const T*)a.hgrad;
    double acc = 0.0;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        T h[9], d[9], s[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            h[c] = hg[c * cs + v];
            d[c] = T(c == a.unit ? 1 : 0);
        }
        const double* m = a.lame + 2 * a.phase[v];
        svk_tangent_apply<T>(h, (T)m[0], (T)m[1], d, s);
#pragma unroll
        for (int c = 0; c < 9; ++c) acc += (double)s[c] * (double)s[c];
    }
    double part[1] = {block_sum(acc)};
    if (!publish_partials<1>(part, a.partials, blockIdx.x, gridDim.x, &a.dev->ticket)) return;
    double tot[1];
    reduce_partials<1>(a.partials, gridDim.x, &a.dev->ticket, tot);
    if (threadIdx.x == 0) a.cg->floor2 = kRoundoffRel * kRoundoffRel * tot[0];
}

// Macroscopic tangent, column `unit`: the voxel sums of K : (E_unit + x),
// x the solution of G K x = -G (K : E_unit); dev->sum[9].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fs_tangent_average(FsPointArgs a) {
    const long long V = a.V, cs = a.cs;
    const T* hg = (const T*)a.hgrad;
    const T* x = (const T*)a.x;
    double acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.0;
    for (long long v = (long long)blockIdx.x * kThreads + threadIdx.x; v < V;
         v += (long long)gridDim.x * kThreads) {
        T h[9], d[9], s[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            h[c] = hg[c * cs + v];
            d[c] = x[c * cs + v] + T(c == a.unit ? 1 : 0);
        }
        const double* m = a.lame + 2 * a.phase[v];
        svk_tangent_apply<T>(h, (T)m[0], (T)m[1], d, s);
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] += (double)s[c];
    }
    double part[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) part[c] = block_sum(acc[c]);
    if (!publish_partials<9>(part, a.partials, blockIdx.x, gridDim.x, &a.dev->ticket)) return;
    double tot[9];
    reduce_partials<9>(a.partials, gridDim.x, &a.dev->ticket, tot);
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int c = 0; c < 9; ++c) a.dev->sum[c] = tot[c];
}

// Loop condition of the device-resident CG graph; stops after `cap` passes
// whatever the solve reports.
__global__ void k_fs_cg_continue(cudaGraphConditionalHandle cond, const CGState* cg, unsigned int* guard,
                                 unsigned int cap) {
    if (threadIdx.x != 0) return;
    bool run = cg->done == CG_RUNNING;
    if (++(*guard) >= cap) run = false;
    cudaGraphSetConditional(cond, run ? 1u : 0u);
}

}  // namespace fftg

using namespace fftg;

namespace {

enum : int {
    FSK_CONSTITUTIVE_F32 = FK_COUNT, FSK_CONSTITUTIVE_F64, FSK_CG_UPDATE_F32, FSK_CG_UPDATE_F64,
    FSK_CG_FINISH_F32, FSK_CG_FINISH_F64, FSK_NEWTON_UPDATE_F32, FSK_NEWTON_UPDATE_F64, FSK_TANGENT_FLOOR,
    FSK_TANGENT_AVERAGE, FSK_CG_RR, FSK_COUNT
};
const char* const kFsKindNames[FSK_COUNT] = {
    "fs_p1_plain_f64", "fs_p1_plain_f32", "fs_p1_tan_f64", "fs_p1_tan_f32", "fs_p1_cg_f64", "fs_p1_cg_f32",
    "fs_p2_f64", "fs_p2_f32", "fs_p3_f64", "fs_p3_f32", "fs_p4_f64", "fs_p4_f32",
    "fs_p5_plain_f64", "fs_p5_plain_f32", "fs_p5_dot_f64", "fs_p5_dot_f32",
    "fs_p5_rhs_f64_to_f64", "fs_p5_rhs_f64_to_f32", "fs_p1_plain_dd", "fs_p2_dd", "fs_p3_dd", "fs_p4_dd",
    "fs_p5_rhs_dd_to_f32", "fs_p5_plain_dd_to_f64", "fs_p1_tanrhs_f64", "fs_p1_tanrhs_f32",
    "fs_p5_rhs_f32_to_f32", "fs_p1_cgf_f32", "fs_p5_cgf_f32",
    "fs_constitutive_f32", "fs_constitutive_f64", "fs_cg_update_f32", "fs_cg_update_f64",
    "fs_cg_finish_f32", "fs_cg_finish_f64", "fs_newton_update_f32", "fs_newton_update_f64",
    "fs_tangent_floor", "fs_tangent_average", "fs_cg_rr_f32"};

// Iterations without a new minimum of <r, r> after which an FP32 inner
// solve counts as stagnated (as in the small-strain driver).
constexpr int kFsStagWindow = 25;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct FsLayout {
    size_t off_phase, off_lame, off_Fstar, off_Fwork, off_P, off_hgrad, off_x, off_r, off_p, off_q,
        off_spec, off_tw32, off_tw64, off_twdd, off_partials, off_cg, off_dev, off_Fbar, off_guard, total;
};

FsLayout fs_layout(int N, bool mixed) {
    const size_t cs = (size_t)comp_stride(N), H = (size_t)(N + 1) / 2;
    const size_t ts = mixed ? 4 : 8;
    const size_t rb = (size_t)std::max(fs_row_blocks(N, true), fs_row_blocks(N, false));
    const size_t npart = std::max((size_t)kFsPointBlocks * 10, rb * 2);
    FsLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.off_phase = take(cs);
    L.off_lame = take(256 * 2 * 8);
    L.off_Fstar = take(9 * cs * 8);
    L.off_Fwork = take(9 * cs * 8);
    L.off_P = take(9 * cs * 8);
    L.off_hgrad = take(9 * cs * ts);
    L.off_x = take(9 * cs * ts);
    L.off_r = take(9 * cs * ts);
    L.off_p = take(9 * cs * ts);
    L.off_q = take(9 * cs * ts);
    L.off_spec = take(9 * (size_t)N * N * H * 16);  // FP64 complex: the residual's size
    L.off_tw32 = take((size_t)N * 8);
    L.off_tw64 = take((size_t)N * 16);
    L.off_twdd = take((size_t)N * 16);
    L.off_partials = take(npart * 8);
    L.off_cg = take(sizeof(CGState));
    L.off_dev = take(sizeof(FsDev));
    L.off_Fbar = take(9 * 8);
    L.off_guard = take(64);
    L.total = o;
    return L;
}

bool fs_options_valid(const fftg_options& o) {
    return (o.precision == FFTG_FP64 || o.precision == FFTG_MIXED) && o.max_newton >= 1 && o.max_cg >= 1 &&
           o.fixed_cg >= 0 && o.fixed_newton >= 0 && o.solver == FFTG_SOLVER_CG && !o.workspace &&
           std::isfinite(o.cg_inner_floor) && o.cg_inner_floor >= 0.0;
}

}  // namespace

struct fftg_fs_handle {
    int N = 0, H = 0;
    long long V = 0, cs = 0;
    int mixed = 1;
    fftg_options opt{};
    cudaStream_t stream = nullptr;
    cudaError_t last_cuda = cudaSuccess;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    uint8_t* phase = nullptr;
    double* lame = nullptr;
    double* Fstar = nullptr;   // committed F*
    double* Fwork = nullptr;   // F* during an increment
    double* P = nullptr;
    void* hgrad = nullptr;     // H = F - I in the inner precision
    void* x = nullptr;
    void* r = nullptr;
    void* p = nullptr;
    void* q = nullptr;
    void* spec = nullptr;
    void* tw32 = nullptr;
    void* tw64 = nullptr;
    void* twdd = nullptr;
    double* partials = nullptr;
    CGState* cg = nullptr;
    FsDev* dev = nullptr;
    double* Fbar_dev = nullptr;
    unsigned int* guard = nullptr;
    CGState* h_cg = nullptr;   // pinned mirrors
    FsDev* h_dev = nullptr;
    double* h_Fbar = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_broken = false;
    double Fbar[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // committed
    bool P_current = false;    // P holds the stress of the committed state
    fftg_stats stats{};
    long long launches = 0;
    // profiling: event pairs drained into per-kind totals
    bool prof_on = false;
    std::vector<cudaEvent_t> ev0, ev1;
    std::vector<int> ev_kind;
    int ev_n = 0;
    double prof_ms[FSK_COUNT] = {};
    long long prof_cnt[FSK_COUNT] = {};
};

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            h->last_cuda = e_;                     \
            return FFTG_ECUDA;                     \
        }                                          \
    } while (0)

namespace {

constexpr int kFsRing = 2048;

cudaError_t fs_prof_drain(fftg_fs_handle* h) {
    if (h->ev_n == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(h->ev1[h->ev_n - 1]);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < h->ev_n; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, h->ev0[i], h->ev1[i]);
        if (e != cudaSuccess) return e;
        h->prof_ms[h->ev_kind[i]] += t;
        h->prof_cnt[h->ev_kind[i]] += 1;
    }
    h->ev_n = 0;
    return cudaSuccess;
}

int fs_prof_begin(fftg_fs_handle* h, int kind) {
    ++h->launches;
    if (!h->prof_on) return -1;
    if (h->ev_n == kFsRing && fs_prof_drain(h) != cudaSuccess) return -1;
    const int i = h->ev_n++;
    h->ev_kind[i] = kind;
    cudaEventRecord(h->ev0[i], h->stream);
    return i;
}

void fs_prof_end(fftg_fs_handle* h, int slot) {
    if (slot >= 0) cudaEventRecord(h->ev1[slot], h->stream);
}

cudaError_t fs_pass(fftg_fs_handle* h, FsPassKind kind, const FsArgs& a) {
    const int slot = fs_prof_begin(h, kind);
    const cudaError_t e = run_fs_pass(h->N, kind, a, h->stream);
    fs_prof_end(h, slot);
    return e;
}

// FFT precision of a pass sequence
enum : int { FFT_F32 = 0, FFT_F64 = 1, FFT_DD = 2 };

// The mixed path's residual G P uses double-float FFTs of the FP64 stress
// (as the small-strain driver does); 0: FP64 FFTs.
#ifndef FFTG_RESIDUAL_DD
#define FFTG_RESIDUAL_DD 1
#endif

FsArgs fs_args(fftg_fs_handle* h, int prec) {
    FsArgs a{};
    a.tw = prec == FFT_DD ? h->twdd : prec == FFT_F64 ? h->tw64 : h->tw32;
    a.partials = h->partials;
    a.cs = h->cs;
    a.phase = h->phase;
    a.lame = h->lame;
    a.hgrad = h->hgrad;
    a.out = h->spec;
    return a;
}

// Every buffer pointer of the handle; kernels read only the ones they use
// (the constitutive kernel takes its inputs and outputs from its caller).
FsPointArgs point_args(fftg_fs_handle* h) {
    FsPointArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.Fbar = h->Fbar_dev;
    u.Fs = h->Fstar;
    u.hgrad = h->hgrad;
    u.phase = h->phase;
    u.lame = h->lame;
    u.dev = h->dev;
    u.partials = h->partials;
    u.x = h->x;
    u.r = h->r;
    u.p = h->p;
    u.q = h->q;
    u.cg = h->cg;
    return u;
}

// Spectrum passes P2, P3 (scale on Ghat), P4.
int fs_p234(fftg_fs_handle* h, int prec, double scale, CGState* cg, const double* red_in = nullptr,
            int red_n = 0) {
    FsArgs a = fs_args(h, prec);
    a.cg = cg;
    a.scale = scale;
    a.red_in = red_in;
    a.red_n = red_n;
    CK(fs_pass(h, prec == FFT_DD ? FK_P2_DD : prec == FFT_F64 ? FK_P2_F64 : FK_P2_F32, a));
    a.red_in = nullptr;
    CK(fs_pass(h, prec == FFT_DD ? FK_P3_DD : prec == FFT_F64 ? FK_P3_F64 : FK_P3_F32, a));
    CK(fs_pass(h, prec == FFT_DD ? FK_P4_DD : prec == FFT_F64 ? FK_P4_F64 : FK_P4_F32, a));
    return FFTG_OK;
}

// P and H at Fbar_dev + F (F = Fwork or Fstar); totals in dev; CG floor.
int fs_constitutive(fftg_fs_handle* h, const double* F, bool write_h, CGState* cg) {
    FsPointArgs u = point_args(h);
    u.Fs = F;
    u.P = h->P;
    u.hgrad = write_h ? h->hgrad : nullptr;
    u.cg = cg;
    const int slot = fs_prof_begin(h, h->mixed ? FSK_CONSTITUTIVE_F32 : FSK_CONSTITUTIVE_F64);
    if (h->mixed)
        k_fs_constitutive<float><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
    else
        k_fs_constitutive<double><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
    fs_prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

// r = -G P (FP64 FFTs, or double-float ones in the mixed path) rounded to
// the inner precision, CG start; x = 0.
int fs_residual(fftg_fs_handle* h) {
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    const int prec = (h->mixed && FFTG_RESIDUAL_DD) ? FFT_DD : FFT_F64;
    FsArgs a = fs_args(h, prec);
    a.in = h->P;
    CK(fs_pass(h, prec == FFT_DD ? FK_P1_PLAIN_DD : FK_P1_PLAIN_F64, a));
    int rc = fs_p234(h, prec, -invN3, nullptr);
    if (rc) return rc;
    FsArgs b = fs_args(h, prec);
    b.in = h->spec;
    b.out = h->r;
    b.cg = h->cg;
    CK(fs_pass(h, prec == FFT_DD ? FK_P5_RHS_DD_TO_F32 : h->mixed ? FK_P5_RHS_F64_TO_F32 : FK_P5_RHS_F64_TO_F64, b));
    CK(cudaMemsetAsync(h->x, 0, 9 * h->cs * (h->mixed ? 4 : 8), h->stream));
    return FFTG_OK;
}

// The mixed path's CG runs without the update pass: alpha from <p, K : p>
// in P1, r -= alpha q in P5 (fs_passes.cuh, FS_P1_CGF). 0: P1 / P5 with
// <p, q> and the update pass, as in the FP64 path.
#ifndef FFTG_FS_CG_FUSED
#define FFTG_FS_CG_FUSED 1
#endif
bool fs_cg_fused(const fftg_fs_handle* h) { return FFTG_FS_CG_FUSED && h->mixed; }

// One CG iteration: P1 (x, p updates and K : p), P2-P4, P5 (q, <p, q>),
// then r -= alpha q; in the mixed path P1 (with <p, K : p>), P2-P4 and P5
// (r -= alpha q, <r, r>).
int fs_cg_iteration(fftg_fs_handle* h) {
    const bool f64 = !h->mixed;
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    const int prec = f64 ? FFT_F64 : FFT_F32;
    if (fs_cg_fused(h)) {
        FsArgs a = fs_args(h, FFT_F32);
        a.aux = h->r;
        a.aux2 = h->p;
        a.aux3 = h->x;
        a.cg = h->cg;
        CK(fs_pass(h, FK_P1_CGF_F32, a));
        // P2 reduces P1's block partials of <p, K : p> (alpha)
        int rc = fs_p234(h, FFT_F32, invN3, h->cg, h->partials, fs_row_blocks(h->N, false));
        if (rc) return rc;
        FsArgs b = fs_args(h, FFT_F32);
        b.in = h->spec;
        b.aux = h->r;
        b.aux3 = h->r;
        b.cg = h->cg;
        CK(fs_pass(h, FK_P5_CGF_F32, b));
        // <r, r> from P5's block partials: beta and the stopping tests
        const int slot = fs_prof_begin(h, FSK_CG_RR);
        k_cg_rr<<<1, 1024, 0, h->stream>>>(h->partials, fs_row_blocks(h->N, false), h->cg);
        fs_prof_end(h, slot);
        CK(cudaGetLastError());
        return FFTG_OK;
    }
    FsArgs a = fs_args(h, prec);
    a.aux = h->r;
    a.aux2 = h->p;
    a.aux3 = h->x;
    a.cg = h->cg;
    CK(fs_pass(h, f64 ? FK_P1_CG_F64 : FK_P1_CG_F32, a));
    int rc = fs_p234(h, prec, invN3, h->cg);
    if (rc) return rc;
    FsArgs b = fs_args(h, prec);
    b.in = h->spec;
    b.out = h->q;
    b.aux = h->p;
    b.cg = h->cg;
    CK(fs_pass(h, f64 ? FK_P5_DOT_F64 : FK_P5_DOT_F32, b));
    FsPointArgs u = point_args(h);
    const int slot = fs_prof_begin(h, f64 ? FSK_CG_UPDATE_F64 : FSK_CG_UPDATE_F32);
    if (f64)
        k_fs_cg_update<double><<<fs_vector_blocks(h->cs, 8), kThreads, 0, h->stream>>>(u);
    else
        k_fs_cg_update<float><<<fs_vector_blocks(h->cs, 4), kThreads, 0, h->stream>>>(u);
    fs_prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

int fs_cg_finish(fftg_fs_handle* h) {
    FsPointArgs u = point_args(h);
    const int slot = fs_prof_begin(h, h->mixed ? FSK_CG_FINISH_F32 : FSK_CG_FINISH_F64);
    if (h->mixed)
        k_fs_cg_finish<float><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
    else
        k_fs_cg_finish<double><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
    fs_prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

void fs_free_graph(fftg_fs_handle* h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
}

// The device-resident CG loop: a graph whose conditional WHILE node repeats
// one iteration while the solve runs (built once per handle: the buffers
// never move).
int fs_build_graph(fftg_fs_handle* h) {
    if (cudaGraphCreate(&h->graph, 0) != cudaSuccess) return FFTG_ECUDA;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, h->graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return FFTG_ECUDA;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &p) != cudaSuccess) return FFTG_ECUDA;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess)
        return FFTG_ECUDA;
    const long long before = h->launches;
    int rc = fs_cg_iteration(h);
    const unsigned int cap = (unsigned int)((h->opt.fixed_cg > 0 ? h->opt.fixed_cg : h->opt.max_cg) + 4);
    if (rc == FFTG_OK) {
        k_fs_cg_continue<<<1, 32, 0, h->stream>>>(cond, h->cg, h->guard, cap);
        if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
    }
    h->launches = before;  // capture enqueues nothing
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(h->stream, &captured) != cudaSuccess || rc) return FFTG_ECUDA;
    if (cudaGraphInstantiate(&h->exec, h->graph, 0) != cudaSuccess) return FFTG_ECUDA;
    return FFTG_OK;
}

// Runs the CG solve to its end: one graph launch, or (profiling, graphs
// off or refused) iterations enqueued from the host in growing chunks.
int fs_run_cg(fftg_fs_handle* h) {
    if (h->opt.cg_graph && !h->prof_on && !h->graph_broken) {
        if (!h->exec && fs_build_graph(h) != FFTG_OK) {
            cudaStreamCaptureStatus cs;
            if (cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(h->stream, &junk);
                if (junk) cudaGraphDestroy(junk);
            }
            fs_free_graph(h);
            cudaGetLastError();
            h->graph_broken = true;
        }
        if (h->exec) {
            CK(cudaMemsetAsync(h->guard, 0, sizeof(unsigned int), h->stream));
            CK(cudaGraphLaunch(h->exec, h->stream));
            int rc = fs_cg_finish(h);
            if (rc) return rc;
            CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            h->launches += 7LL * (h->h_cg->it + 1);  // one of each per loop pass
            return FFTG_OK;
        }
    }
    CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int chunk = 2, launched = 0;
    const int cap = (h->opt.fixed_cg > 0 ? h->opt.fixed_cg : h->opt.max_cg) + 1;
    while (h->h_cg->done == CG_RUNNING) {
        if (launched > cap) return FFTG_ENOCONV_CG;  // defensive: should not happen
        for (int k = 0; k < chunk; ++k) {
            int rc = fs_cg_iteration(h);
            if (rc) return rc;
        }
        launched += chunk;
        chunk = std::min(chunk * 2, 16);
        CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return fs_cg_finish(h);
}

// Mixed precision: x <- G x in FP32 after each solve (the FP32 recursion
// lets x drift out of the compatible space; see the small-strain driver).
int fs_project_solution(fftg_fs_handle* h) {
    if (!h->mixed) return FFTG_OK;
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    FsArgs a = fs_args(h, FFT_F32);
    a.in = h->x;
    CK(fs_pass(h, FK_P1_PLAIN_F32, a));
    int rc = fs_p234(h, FFT_F32, invN3, nullptr);
    if (rc) return rc;
    FsArgs b = fs_args(h, FFT_F32);
    b.in = h->spec;
    b.out = h->x;
    CK(fs_pass(h, FK_P5_PLAIN_F32, b));
    return FFTG_OK;
}

void fs_set_cg(fftg_fs_handle* h, double tol) {
    CGState& c = *h->h_cg;
    std::memset(&c, 0, sizeof(CGState));
    c.tol2 = tol * tol;
    c.max_it = h->opt.max_cg;
    c.fixed_it = h->opt.fixed_cg;
    c.stag_window = (h->mixed && h->opt.fixed_cg <= 0) ? kFsStagWindow : 0;
    c.done = CG_RUNNING;
}

// Copy a [9][V] field between the caller layout (stride V) and the padded
// one (stride cs).
cudaError_t fs_copy(fftg_fs_handle* h, void* dst, bool dst_padded, const void* src, bool src_padded, size_t elem,
                    cudaMemcpyKind kind) {
    const size_t w = (size_t)h->V * elem;
    const size_t dp = (dst_padded ? (size_t)h->cs : (size_t)h->V) * elem;
    const size_t sp = (src_padded ? (size_t)h->cs : (size_t)h->V) * elem;
    return cudaMemcpy2DAsync(dst, dp, src, sp, w, 9, kind, h->stream);
}

int fs_upload_Fbar(fftg_fs_handle* h, const double F[9]) {
    std::memcpy(h->h_Fbar, F, 9 * sizeof(double));
    CK(cudaMemcpyAsync(h->Fbar_dev, h->h_Fbar, 9 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    return FFTG_OK;
}

}  // namespace

// ---------------------------------------------------------------- public API
extern "C" {

int fftg_fs_workspace_size(int N, const fftg_options* opt, size_t* bytes) {
    if (!bytes || !supported_grid(N)) return FFTG_EINVAL;
    fftg_options o;
    if (opt) o = *opt; else fftg_default_options(&o);
    if (o.precision != FFTG_FP64 && o.precision != FFTG_MIXED) return FFTG_EINVAL;
    *bytes = fs_layout(N, o.precision == FFTG_MIXED).total;
    return FFTG_OK;
}

void fftg_fs_destroy(fftg_fs_handle* h) {
    if (!h) return;
    if (h->stream || h->ws) cudaStreamSynchronize(h->stream);
    fs_free_graph(h);
    for (size_t i = 0; i < h->ev0.size(); ++i) {
        if (h->ev0[i]) cudaEventDestroy(h->ev0[i]);
        if (h->ev1[i]) cudaEventDestroy(h->ev1[i]);
    }
    if (h->ws) cudaFree(h->ws);
    if (h->h_cg) cudaFreeHost(h->h_cg);
    if (h->h_dev) cudaFreeHost(h->h_dev);
    if (h->h_Fbar) cudaFreeHost(h->h_Fbar);
    delete h;
}

int fftg_fs_create(fftg_fs_handle** out, int N, const uint8_t* phase, int nphase, const fftg_svk_phase* mats,
                   const fftg_options* opt) {
    if (!out || !phase || !mats || nphase < 1 || nphase > 256 || !supported_grid(N)) return FFTG_EINVAL;
    *out = nullptr;
    fftg_options o;
    if (opt) o = *opt; else fftg_default_options(&o);
    if (!fs_options_valid(o)) return FFTG_EINVAL;
    for (int i = 0; i < nphase; ++i)
        if (!(std::isfinite(mats[i].lambda) && mats[i].lambda >= 0.0 && std::isfinite(mats[i].mu) &&
              mats[i].mu > 0.0))
            return FFTG_EINVAL;
    const size_t V = (size_t)N * N * N;
    for (size_t v = 0; v < V; ++v)
        if (phase[v] >= nphase) return FFTG_EINVAL;
    fftg_fs_handle* h = new (std::nothrow) fftg_fs_handle();
    if (!h) return FFTG_ENOMEM;
    h->N = N;
    h->H = (N + 1) / 2;
    h->V = (long long)V;
    h->cs = comp_stride(N);
    h->mixed = o.precision == FFTG_MIXED;
    h->opt = o;
    h->stream = (cudaStream_t)o.stream;
    const FsLayout L = fs_layout(N, h->mixed);
    if (cudaMalloc((void**)&h->ws, L.total) != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        fftg_fs_destroy(h);
        return FFTG_ENOMEM;
    }
    h->ws_bytes = L.total;
    h->phase = (uint8_t*)(h->ws + L.off_phase);
    h->lame = (double*)(h->ws + L.off_lame);
    h->Fstar = (double*)(h->ws + L.off_Fstar);
    h->Fwork = (double*)(h->ws + L.off_Fwork);
    h->P = (double*)(h->ws + L.off_P);
    h->hgrad = h->ws + L.off_hgrad;
    h->x = h->ws + L.off_x;
    h->r = h->ws + L.off_r;
    h->p = h->ws + L.off_p;
    h->q = h->ws + L.off_q;
    h->spec = h->ws + L.off_spec;
    h->tw32 = h->ws + L.off_tw32;
    h->tw64 = h->ws + L.off_tw64;
    h->twdd = h->ws + L.off_twdd;
    h->partials = (double*)(h->ws + L.off_partials);
    h->cg = (CGState*)(h->ws + L.off_cg);
    h->dev = (FsDev*)(h->ws + L.off_dev);
    h->Fbar_dev = (double*)(h->ws + L.off_Fbar);
    h->guard = (unsigned int*)(h->ws + L.off_guard);
    if (cudaMallocHost((void**)&h->h_cg, sizeof(CGState)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_dev, sizeof(FsDev)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_Fbar, 9 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        fftg_fs_destroy(h);
        return FFTG_ENOMEM;
    }
    std::vector<double> tw64(2 * N), lame(2 * nphase);
    std::vector<float> tw32(2 * N), twdd(4 * N);
    twiddles(N, tw64.data(), tw32.data(), twdd.data());
    for (int i = 0; i < nphase; ++i) {
        lame[2 * i] = mats[i].lambda;
        lame[2 * i + 1] = mats[i].mu;
    }
    const double I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    std::memcpy(h->h_Fbar, I9, sizeof(I9));
    cudaStream_t s = h->stream;
    if (cudaMemsetAsync(h->ws, 0, L.total, s) != cudaSuccess ||
        cudaMemcpyAsync(h->phase, phase, V, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->lame, lame.data(), lame.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->tw64, tw64.data(), tw64.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->tw32, tw32.data(), tw32.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->twdd, twdd.data(), twdd.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->Fbar_dev, h->h_Fbar, 9 * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        h->last_cuda = cudaGetLastError();
        fftg_fs_destroy(h);
        return FFTG_ECUDA;
    }
    h->ev0.assign(kFsRing, nullptr);
    h->ev1.assign(kFsRing, nullptr);
    h->ev_kind.assign(kFsRing, 0);
    *out = h;
    return FFTG_OK;
}

int fftg_fs_step(fftg_fs_handle* h, const double dF[9], double tol_newton, double tol_cg, double P_out[9],
                 int* newton_iters, int* cg_iters) {
    if (!h || !dF || !P_out || !(tol_newton > 0) || !(tol_cg > 0)) return FFTG_EINVAL;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(dF[k])) return FFTG_ENAN;
    std::memset(&h->stats, 0, sizeof(fftg_stats));
    const double tol_inner = h->mixed ? std::max(tol_cg, h->opt.cg_inner_floor) : tol_cg;
    double Ft[9], nH2 = 0.0;
    for (int k = 0; k < 9; ++k) {
        Ft[k] = h->Fbar[k] + dF[k];
        const double hk = Ft[k] - ((k % 4 == 0) ? 1.0 : 0.0);
        nH2 += hk * hk;
    }
    const double normH = std::sqrt((double)h->V * nH2);
    int rc = fs_upload_Fbar(h, Ft);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->Fwork, h->Fstar, 9 * h->cs * 8, cudaMemcpyDeviceToDevice, h->stream));
    h->P_current = false;
    int it = 0, status = FFTG_OK;
    for (;;) {
        fs_set_cg(h, tol_inner);
        CK(cudaMemcpyAsync(h->cg, h->h_cg, sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
        if ((rc = fs_constitutive(h, h->Fwork, true, h->cg)) || (rc = fs_residual(h)) || (rc = fs_run_cg(h)) ||
            (rc = fs_project_solution(h)))
            break;
        FsPointArgs u = point_args(h);
        u.Fw = h->Fwork;
        const int slot = fs_prof_begin(h, h->mixed ? FSK_NEWTON_UPDATE_F32 : FSK_NEWTON_UPDATE_F64);
        if (h->mixed)
            k_fs_newton_update<float><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        else
            k_fs_newton_update<double><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        fs_prof_end(h, slot);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(h->h_dev, h->dev, sizeof(FsDev), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        const CGState& c = *h->h_cg;
        const double nde = std::sqrt(h->h_dev->de2);
        const double rel = normH > 0 ? nde / normH : (nde == 0 ? 0.0 : INFINITY);
        fftg_stats& st = h->stats;
        if (it < FFTG_MAX_NEWTON_LOG) {
            st.cg_per_newton[it] = c.it;
            st.newton_norm[it] = rel;
            st.residual[it] = h->h_dev->p2 > 0 ? std::sqrt(c.gs2 / h->h_dev->p2) : 0.0;
            st.cg_relres[it] = c.rr0 > 0 ? std::sqrt(c.rr / c.rr0) : 0.0;
            st.cg_status[it] = c.done;
        }
        st.cg_iters += c.it;
        st.newton_iters = ++it;
        if (c.done == CG_BREAKDOWN || !std::isfinite(rel)) {
            status = FFTG_ENAN;
            break;
        }
        if (h->opt.fixed_newton > 0) {
            if (it >= h->opt.fixed_newton) break;
            continue;
        }
        if (rel <= tol_newton || nde == 0.0) break;
        if (it >= h->opt.max_newton) {
            status = FFTG_ENOCONV_NEWTON;
            break;
        }
    }
    if (rc) status = rc;
    h->stats.status = status;
    if (newton_iters) *newton_iters = it;
    if (cg_iters) *cg_iters = h->stats.cg_iters;
    if (status != FFTG_OK) {
        rc = fs_upload_Fbar(h, h->Fbar);  // back to the committed Fbar
        if (rc == FFTG_OK) cudaStreamSynchronize(h->stream);
        return status;
    }
    // stress at the converged state, homogenised; commit
    if ((rc = fs_constitutive(h, h->Fwork, false, nullptr))) return rc;
    CK(cudaMemcpyAsync(h->h_dev, h->dev, sizeof(FsDev), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->Fstar, h->Fwork, 9 * h->cs * 8, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 9; ++k) {
        P_out[k] = h->h_dev->sum[k] / (double)h->V;
        h->Fbar[k] = Ft[k];
    }
    h->P_current = true;
    return FFTG_OK;
}

int fftg_fs_tangent(fftg_fs_handle* h, double tol_cg, double C_out[81], int* cg_iters) {
    if (!h || !C_out || !(tol_cg > 0)) return FFTG_EINVAL;
    const bool f64 = !h->mixed;
    const int prec = f64 ? FFT_F64 : FFT_F32;
    const double tol_inner = h->mixed ? std::max(tol_cg, h->opt.cg_inner_floor) : tol_cg;
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    // tangent data H at the committed state
    int rc = fs_upload_Fbar(h, h->Fbar);
    if (rc) return rc;
    if ((rc = fs_constitutive(h, h->Fstar, true, nullptr))) return rc;
    h->P_current = true;
    int total = 0;
    for (int unit = 0; unit < 9; ++unit) {
        fs_set_cg(h, tol_inner);
        CK(cudaMemcpyAsync(h->cg, h->h_cg, sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
        FsPointArgs u = point_args(h);
        u.unit = unit;
        int slot = fs_prof_begin(h, FSK_TANGENT_FLOOR);
        if (f64)
            k_fs_tangent_floor<double><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        else
            k_fs_tangent_floor<float><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        fs_prof_end(h, slot);
        CK(cudaGetLastError());
        // r = -G (K : E_unit) in the inner precision; CG start; x = 0
        FsArgs a = fs_args(h, prec);
        a.unit = unit;
        CK(fs_pass(h, f64 ? FK_P1_TANRHS_F64 : FK_P1_TANRHS_F32, a));
        if ((rc = fs_p234(h, prec, -invN3, nullptr))) return rc;
        FsArgs b = fs_args(h, prec);
        b.in = h->spec;
        b.out = h->r;
        b.cg = h->cg;
        CK(fs_pass(h, f64 ? FK_P5_RHS_F64_TO_F64 : FK_P5_RHS_F32_TO_F32, b));
        CK(cudaMemsetAsync(h->x, 0, 9 * h->cs * (f64 ? 8 : 4), h->stream));
        if ((rc = fs_run_cg(h)) || (rc = fs_project_solution(h))) return rc;
        if (h->h_cg->done == CG_BREAKDOWN) return FFTG_ENAN;
        total += h->h_cg->it;
        slot = fs_prof_begin(h, FSK_TANGENT_AVERAGE);
        if (f64)
            k_fs_tangent_average<double><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        else
            k_fs_tangent_average<float><<<fs_point_blocks(h->V), kThreads, 0, h->stream>>>(u);
        fs_prof_end(h, slot);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h->h_dev, h->dev, sizeof(FsDev), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int r = 0; r < 9; ++r) C_out[9 * r + unit] = h->h_dev->sum[r] / (double)h->V;
    }
    if (cg_iters) *cg_iters = total;
    return FFTG_OK;
}

int fftg_fs_last_stats(fftg_fs_handle* h, fftg_stats* out) {
    if (!h || !out) return FFTG_EINVAL;
    *out = h->stats;
    return FFTG_OK;
}

int fftg_fs_get_field(fftg_fs_handle* h, int which, double* host_out) {
    if (!h || !host_out) return FFTG_EINVAL;
    if (which == FFTG_FS_FIELD_DEFGRAD) {
        CK(fs_copy(h, host_out, false, h->Fstar, true, 8, cudaMemcpyDeviceToHost));
        CK(cudaStreamSynchronize(h->stream));
        for (int c = 0; c < 9; ++c)
            for (long long v = 0; v < h->V; ++v) host_out[c * h->V + v] += h->Fbar[c];
        return FFTG_OK;
    }
    if (which == FFTG_FS_FIELD_STRESS) {
        if (!h->P_current) {
            int rc = fs_upload_Fbar(h, h->Fbar);  // the committed Fbar
            if (rc == FFTG_OK) rc = fs_constitutive(h, h->Fstar, false, nullptr);
            if (rc) return rc;
            h->P_current = true;
        }
        CK(fs_copy(h, host_out, false, h->P, true, 8, cudaMemcpyDeviceToHost));
        CK(cudaStreamSynchronize(h->stream));
        return FFTG_OK;
    }
    return FFTG_EINVAL;
}

size_t fftg_fs_state_bytes(const fftg_fs_handle* h) {
    return h ? (size_t)(9 + 9 * h->V) * sizeof(double) : 0;
}

int fftg_fs_get_state(fftg_fs_handle* h, void* host_buf, size_t bytes) {
    if (!h || !host_buf || bytes != fftg_fs_state_bytes(h)) return FFTG_EINVAL;
    double* d = (double*)host_buf;
    std::memcpy(d, h->Fbar, 9 * sizeof(double));
    CK(fs_copy(h, d + 9, false, h->Fstar, true, 8, cudaMemcpyDeviceToHost));
    CK(cudaStreamSynchronize(h->stream));
    return FFTG_OK;
}

int fftg_fs_set_state(fftg_fs_handle* h, const void* host_buf, size_t bytes) {
    if (!h || !host_buf || bytes != fftg_fs_state_bytes(h)) return FFTG_EINVAL;
    const double* d = (const double*)host_buf;
    for (size_t k = 0; k < 9 + 9 * (size_t)h->V; ++k)
        if (!std::isfinite(d[k])) return FFTG_EINVAL;
    CK(fs_copy(h, h->Fstar, true, d + 9, false, 8, cudaMemcpyHostToDevice));
    int rc = fs_upload_Fbar(h, d);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(h->Fbar, d, 9 * sizeof(double));
    h->P_current = false;
    return FFTG_OK;
}

int fftg_fs_op_project(fftg_fs_handle* h, int precision, const void* A_dev, void* out_dev) {
    if (!h || !A_dev || !out_dev || (precision != FFTG_FP64 && precision != FFTG_MIXED && precision != FFTG_DD))
        return FFTG_EINVAL;
    const int prec = precision == FFTG_FP64 ? FFT_F64 : precision == FFTG_DD ? FFT_DD : FFT_F32;
    const bool f64 = prec != FFT_F32;  // FP64 buffers (FFTG_FP64, FFTG_DD)
    const size_t el = f64 ? 8 : 4;
    // staged through the padded buffer P (FP64) or x (FP32)
    void* buf = f64 ? (void*)h->P : h->x;
    if (!f64 && !h->mixed) return FFTG_EINVAL;  // FP32 buffers exist only in a mixed handle
    h->P_current = false;
    CK(fs_copy(h, buf, true, A_dev, false, el, cudaMemcpyDeviceToDevice));
    FsArgs a = fs_args(h, prec);
    a.in = buf;
    CK(fs_pass(h, prec == FFT_DD ? FK_P1_PLAIN_DD : f64 ? FK_P1_PLAIN_F64 : FK_P1_PLAIN_F32, a));
    int rc = fs_p234(h, prec, 1.0 / ((double)h->N * h->N * h->N), nullptr);
    if (rc) return rc;
    FsArgs b = fs_args(h, prec);
    b.in = h->spec;
    b.out = buf;
    CK(fs_pass(h, prec == FFT_DD ? FK_P5_PLAIN_DD_TO_F64 : f64 ? FK_P5_PLAIN_F64 : FK_P5_PLAIN_F32, b));
    CK(fs_copy(h, out_dev, false, buf, true, el, cudaMemcpyDeviceToDevice));
    return FFTG_OK;
}

int fftg_fs_op_matvec(fftg_fs_handle* h, int precision, const void* p_dev, void* q_dev, double* pq) {
    if (!h || !p_dev || !q_dev || (precision != FFTG_FP64 && precision != FFTG_MIXED)) return FFTG_EINVAL;
    const bool f64 = precision == FFTG_FP64;
    if (f64 == (bool)h->mixed) return FFTG_EINVAL;  // the handle's inner precision
    const size_t el = f64 ? 8 : 4;
    // tangent data H at the committed state
    int rc = fs_upload_Fbar(h, h->Fbar);
    if (rc) return rc;
    if ((rc = fs_constitutive(h, h->Fstar, true, nullptr))) return rc;
    h->P_current = true;
    CK(fs_copy(h, h->p, true, p_dev, false, el, cudaMemcpyDeviceToDevice));
    const int prec = f64 ? FFT_F64 : FFT_F32;
    FsArgs a = fs_args(h, prec);
    a.in = h->p;
    CK(fs_pass(h, f64 ? FK_P1_TAN_F64 : FK_P1_TAN_F32, a));
    if ((rc = fs_p234(h, prec, 1.0 / ((double)h->N * h->N * h->N), nullptr))) return rc;
    // <p, q> through the DOT pass on a scratch CG state
    fs_set_cg(h, 1.0);
    CK(cudaMemcpyAsync(h->cg, h->h_cg, sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
    FsArgs b = fs_args(h, prec);
    b.in = h->spec;
    b.out = h->q;
    b.aux = h->p;
    b.cg = h->cg;
    CK(fs_pass(h, f64 ? FK_P5_DOT_F64 : FK_P5_DOT_F32, b));
    CK(fs_copy(h, q_dev, false, h->q, true, el, cudaMemcpyDeviceToDevice));
    if (pq) {
        CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *pq = h->h_cg->pq;
    }
    return FFTG_OK;
}

int fftg_fs_profile_kinds(void) { return FSK_COUNT; }

const char* fftg_fs_profile_name(int kind) { return (kind >= 0 && kind < FSK_COUNT) ? kFsKindNames[kind] : nullptr; }

int fftg_fs_profile_enable(fftg_fs_handle* h, int on) {
    if (!h) return FFTG_EINVAL;
    if (on && !h->ev0[0]) {
        for (int i = 0; i < kFsRing; ++i)
            if (cudaEventCreate(&h->ev0[i]) != cudaSuccess || cudaEventCreate(&h->ev1[i]) != cudaSuccess) {
                h->last_cuda = cudaGetLastError();
                return FFTG_ECUDA;
            }
    }
    if (!on) CK(fs_prof_drain(h));
    h->prof_on = on != 0;
    std::fill(h->prof_ms, h->prof_ms + FSK_COUNT, 0.0);
    std::fill(h->prof_cnt, h->prof_cnt + FSK_COUNT, 0LL);
    return FFTG_OK;
}

int fftg_fs_profile_read(fftg_fs_handle* h, int kind, double* total_ms, long long* launches) {
    if (!h || kind < 0 || kind >= FSK_COUNT) return FFTG_EINVAL;
    CK(fs_prof_drain(h));
    if (total_ms) *total_ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_cnt[kind];
    return FFTG_OK;
}

long long fftg_fs_launch_count(const fftg_fs_handle* h) { return h ? h->launches : 0; }

}  // extern "C"
