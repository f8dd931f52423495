// C-ABI of the fftg library: handle lifetime, the Newton-CG driver of
// Algorithm 1 over a batch of cells, and the operator-level entry points.
// Everything numerical runs in the kernels of passes.cuh and pointwise.cuh;
// the host only sequences launches and reads a few scalars per Newton
// iteration. A handle holds B >= 1 cells of the same grid: every launch
// covers all of them, each cell with its own CG and Newton state, and an
// active mask lets cells join and leave between Newton iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fftg.h"
#include "driver.h"
#include "host_common.h"
#include "materials.h"
#include "passes.cuh"
#include "pointwise.cuh"
#include "schedule.cuh"
#include "batch.cuh"

namespace fftg {
#define FFTG_EXTERN_N(n) extern template cudaError_t run_pass_n<n>(PassKind, const PassArgs&, int, cudaStream_t);
FFTG_EXTERN_N(3)
FFTG_EXTERN_N(5)
FFTG_EXTERN_N(9)
FFTG_EXTERN_N(15)
FFTG_EXTERN_N(25)
FFTG_EXTERN_N(27)
FFTG_EXTERN_N(45)
FFTG_EXTERN_N(75)
FFTG_EXTERN_N(81)
FFTG_EXTERN_N(125)
FFTG_EXTERN_N(135)
FFTG_EXTERN_N(225)
FFTG_EXTERN_N(243)
#undef FFTG_EXTERN_N

static bool supported_n(int N) { return supported_grid(N); }

cudaError_t run_pass(int N, PassKind kind, const PassArgs& a, int nf, cudaStream_t s) {
    const int tk = tuned_kind(kind);
    if (tk >= 0) {
        const int v = schedule_variant(N, tk);
        if (v > 0) return run_variant(N, tk, v, a, nf, s);
    }
    switch (N) {
#define FFTG_CASE(n) case n: return run_pass_n<n>(kind, a, nf, s);
        FFTG_CASE(3) FFTG_CASE(5) FFTG_CASE(9) FFTG_CASE(15) FFTG_CASE(25) FFTG_CASE(27)
        FFTG_CASE(45) FFTG_CASE(75) FFTG_CASE(81) FFTG_CASE(125) FFTG_CASE(135) FFTG_CASE(225)
        FFTG_CASE(243)
#undef FFTG_CASE
        default: return cudaErrorInvalidValue;
    }
}

// FP32: the most blocks of any schedule variant of the row passes (half the
// rows per block), so that the partial-sum buffer fits every schedule.
template <int N>
static int row_blocks_n(bool fp64) {
    return fp64 ? Cfg<N, double>::row_blocks
                : std::max(Cfg<N, float>::row_blocks, Cfg<N, float, Plan<N>::N1, 1>::row_blocks);
}

int row_blocks(int N, bool fp64) {
    switch (N) {
#define FFTG_CASE(n) case n: return row_blocks_n<n>(fp64);
        FFTG_CASE(3) FFTG_CASE(5) FFTG_CASE(9) FFTG_CASE(15) FFTG_CASE(25) FFTG_CASE(27)
        FFTG_CASE(45) FFTG_CASE(75) FFTG_CASE(81) FFTG_CASE(125) FFTG_CASE(135) FFTG_CASE(225)
        FFTG_CASE(243)
#undef FFTG_CASE
        default: return 0;
    }
}
}  // namespace fftg

using namespace fftg;

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            h->last_cuda = e_;                     \
            return FFTG_ECUDA;                     \
        }                                          \
    } while (0)

namespace {
enum : int {
    KK_CONSTITUTIVE_F32 = PK_COUNT, KK_CONSTITUTIVE_F64, KK_CG_UPDATE_F32, KK_CG_UPDATE_F64,
    KK_NEWTON_UPDATE_F32, KK_NEWTON_UPDATE_F64, KK_TANGENT_FLOOR, KK_TANGENT_AVERAGE,
    KK_CG_FINISH_F32, KK_CG_FINISH_F64, KK_TANGENT_BOUNDS, KK_CG_RR, KK_COUNT
};
const char* const kKindNames[KK_COUNT] = {
    "p1_plain_f64", "p1_plain_f32", "p1_tan_f64", "p1_tan_f32", "p1_cg_f64", "p1_cg_f32",
    "p1_tanrhs_f64", "p1_tanrhs_f32", "p2_f64", "p2_f32", "p4_f64", "p4_f32", "p3_f64", "p3_f32",
    "p5_plain_f64", "p5_plain_f32", "p5_dot_f64", "p5_dot_f32", "p5_rhs_f64_to_f64",
    "p5_rhs_f64_to_f32", "p5_rhs_f32_to_f32", "p1_plain_dd", "p2_dd", "p3_dd", "p4_dd",
    "p5_rhs_dd_to_f32", "p5_plain_dd_to_f64", "p1_cgf_f32", "p5_cgf_f32", "constitutive_f32",
    "constitutive_f64",
    "cg_update_f32", "cg_update_f64", "newton_update_f32", "newton_update_f64", "tangent_floor",
    "tangent_average", "cg_finish_f32", "cg_finish_f64", "tangent_bounds", "cg_rr_f32"};

// Ring of event pairs around the handle's launches; drained at every read.
struct Prof {
    static constexpr int kRing = 4096;
    bool on = false;
    cudaEvent_t ev0[kRing] = {}, ev1[kRing] = {};
    int kind[kRing] = {};
    int n = 0;
    double ms[KK_COUNT] = {};
    long long cnt[KK_COUNT] = {};
};

// Iterations without a new minimum of <r, r> after which an FP32 inner
// solve is considered stagnated.
constexpr int kStagWindow = 25;
}  // namespace

struct fftg_handle {
    int N = 0;
    long long V = 0;
    long long cs = 0;            // component stride of the fields (padded)
    int H = 0;
    int mixed = 1;
    int nrhs = 6;
    int B = 1;                   // cells
    int nf = 6;                  // CG fields held: max(B, nrhs)
    int sel = 0;                 // cell addressed by the single-cell calls
    fftg_options opt{};
    cudaStream_t stream = nullptr;
    cudaError_t last_cuda = cudaSuccess;
    bool own_ws = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;

    uint8_t* phase = nullptr;    // [B][cs]
    double* mats = nullptr;
    int nphase = 0;
    double* eps_star = nullptr;  // [B][6][cs] committed
    double* eps_work = nullptr;  // [B][6][cs] trial during an increment
    double* eps_p = nullptr;     // [B][6][cs] committed
    double* eps_p_tr = nullptr;  // [B][6][cs] trial
    double* epbar = nullptr;     // [B][cs] committed
    double* epbar_tr = nullptr;  // [B][cs] trial
    double* sigma = nullptr;     // [B][6][cs]
    void* tangent = nullptr;     // [B][7][cs] inner precision
    void* x = nullptr;           // [nf][6][cs] inner precision
    void* r = nullptr;
    void* p = nullptr;
    void* q = nullptr;
    void* spec = nullptr;
    void* tw32 = nullptr;
    void* tw64 = nullptr;
    void* twdd = nullptr;
    double* partials = nullptr;
    CGState* cg = nullptr;       // [nf]
    NewtonDev* nd = nullptr;     // [B]
    double* Edev = nullptr;      // [B][6]
    int* active = nullptr;       // [B]
    double* out36 = nullptr;

    CGState* h_cg = nullptr;     // pinned mirrors
    NewtonDev* h_nd = nullptr;
    double* h_out36 = nullptr;
    double* h_E = nullptr;
    int* h_active = nullptr;

    unsigned int* guard = nullptr;   // loop-pass counters: [0] CG graph, [1] Newton loop of a group graph
    int* run_dev = nullptr;          // device-driven increments (fftg_group_step)
    double* dE_dev = nullptr;
    double* Ecom_dev = nullptr;
    int* fin_dev = nullptr;
    IncDev* inc_dev = nullptr;
    struct CgGraph {
        int nf = 0;
        const void* tangent = nullptr;
        long long tstride = 0;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;
    };
    std::vector<CgGraph> graphs;     // small cache of instantiated CG graphs
    unsigned long long graph_clock = 0;
    bool graphs_broken = false;      // the CUDA driver refused: use the chunked path

    std::vector<double> E;           // [B][6] committed
    std::vector<char> have_tangent;  // [B] a converged increment's tangent is held
    std::vector<char> have_update;   // [B] some stress update wrote the tangent
    std::vector<fftg_stats> stats;   // [B]
    long long launches = 0;
    Prof* prof = nullptr;
};

// Drain the recorded event pairs into the per-kind totals.
static cudaError_t prof_drain(fftg_handle* h) {
    Prof* P = h->prof;
    if (!P || P->n == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(P->ev1[P->n - 1]);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < P->n; ++i) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, P->ev0[i], P->ev1[i]);
        if (e != cudaSuccess) return e;
        P->ms[P->kind[i]] += t;
        P->cnt[P->kind[i]] += 1;
    }
    P->n = 0;
    return cudaSuccess;
}

// Bracket one launch: returns the slot to close, or -1 when profiling is off.
static int prof_begin(fftg_handle* h, int kind) {
    ++h->launches;
    Prof* P = h->prof;
    if (!P || !P->on) return -1;
    if (P->n == Prof::kRing && prof_drain(h) != cudaSuccess) return -1;
    const int i = P->n++;
    P->kind[i] = kind;
    cudaEventRecord(P->ev0[i], h->stream);
    return i;
}

static void prof_end(fftg_handle* h, int slot) {
    if (slot >= 0) cudaEventRecord(h->prof->ev1[slot], h->stream);
}

// One pass launch, instrumented.
static cudaError_t pass(fftg_handle* h, PassKind kind, const PassArgs& a, int nf) {
    const int slot = prof_begin(h, kind);
    cudaError_t e = run_pass(h->N, kind, a, nf, h->stream);
    prof_end(h, slot);
    return e;
}

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
    size_t off_phase, off_mats, off_eps_star, off_eps_work, off_eps_p, off_eps_p_tr, off_epbar,
        off_epbar_tr, off_sigma, off_tangent, off_x, off_r, off_p, off_q, off_spec, off_tw32,
        off_tw64, off_twdd, off_partials, off_cg, off_nd, off_E, off_active, off_out36, off_guard, off_run,
        off_dE, off_Ecom, off_fin, off_inc, total;
};

Layout make_layout(int N, int mixed, int nrhs, int B) {
    const size_t cs = (size_t)comp_stride(N);
    const size_t H = (size_t)(N + 1) / 2;
    const size_t ts = mixed ? 4 : 8;
    const size_t nf = (size_t)std::max(B, std::max(1, nrhs));
    const size_t spec1 = 6 * (size_t)N * N * H;  // complex elements per field
    const size_t spec = std::max((size_t)B * spec1 * 16, nf * spec1 * 2 * ts);
    const size_t rb = (size_t)std::max(fftg::row_blocks(N, true), fftg::row_blocks(N, false));
    const size_t npart = std::max({(size_t)kMaxPointwiseBlocks * 36, rb * 2 * nf,
                                   (size_t)B * kMaxPointwiseBlocks * 7, nf * 2432});
    const size_t Bs = (size_t)B;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.off_phase = take(Bs * cs);
    L.off_mats = take(256 * fftg::kMatStride * 8);
    L.off_eps_star = take(Bs * 6 * cs * 8);
    L.off_eps_work = take(Bs * 6 * cs * 8);
    L.off_eps_p = take(Bs * 6 * cs * 8);
    L.off_eps_p_tr = take(Bs * 6 * cs * 8);
    L.off_epbar = take(Bs * cs * 8);
    L.off_epbar_tr = take(Bs * cs * 8);
    L.off_sigma = take(Bs * 6 * cs * 8);
    L.off_tangent = take(Bs * 7 * cs * ts);
    L.off_x = take(nf * 6 * cs * ts);
    L.off_r = take(nf * 6 * cs * ts);
    L.off_p = take(nf * 6 * cs * ts);
    L.off_q = take(nf * 6 * cs * ts);
    L.off_spec = take(spec);
    L.off_tw32 = take((size_t)N * 8);
    L.off_tw64 = take((size_t)N * 16);
    L.off_twdd = take((size_t)N * 16);
    L.off_partials = take(npart * 8);
    L.off_cg = take(nf * sizeof(CGState));
    L.off_nd = take(Bs * sizeof(NewtonDev));
    L.off_E = take(Bs * 6 * 8);
    L.off_active = take(Bs * 4);
    L.off_out36 = take(36 * 8);
    L.off_guard = take(64);
    // device-driven increments (fftg_group_step): per cell run mask, dE,
    // committed E, finish mask and increment state
    L.off_run = take(Bs * 4);
    L.off_dE = take(Bs * 6 * 8);
    L.off_Ecom = take(Bs * 6 * 8);
    L.off_fin = take(Bs * 4);
    L.off_inc = take(Bs * sizeof(IncDev));
    L.total = o;
    return L;
}

bool valid_grid(int N) {
    if (N < 3 || N % 2 == 0) return false;
    int m = N;
    while (m % 3 == 0) m /= 3;
    while (m % 5 == 0) m /= 5;
    return m == 1 && fftg::supported_n(N);
}

double frob6(const double* v) {
    return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] +
                     2.0 * (v[3] * v[3] + v[4] * v[4] + v[5] * v[5]));
}

}  // namespace

// ---------------------------------------------------------------- internals
// FFT precision of a pass sequence
enum : int { FFT_F32 = 0, FFT_F64 = 1, FFT_DD = 2 };

// The mixed path computes its residual G sigma with double-float FFTs
// (dd.cuh) in place of FP64 ones: about 1e-14 of ||sigma|| where FP64 gives
// 1e-16, far below the CG roundoff floor, at a fraction of the FP64 cost on
// this GPU. 0: FP64 FFTs.
#ifndef FFTG_RESIDUAL_DD
#define FFTG_RESIDUAL_DD 1
#endif

static PassArgs base_args(fftg_handle* h, bool fp64) {
    PassArgs a{};
    a.tw = fp64 ? h->tw64 : h->tw32;
    a.partials = h->partials;
    a.cs = h->cs;
    a.fstride = 6 * h->cs;
    a.sstride = 6LL * h->N * h->N * h->H;
    a.tstride = 0;
    return a;
}

// Copy a [6][V] field between a caller layout (component stride V) and the
// padded internal layout (component stride cs).
static cudaError_t copy_field(fftg_handle* h, void* dst, bool dst_padded, const void* src,
                              bool src_padded, size_t elem, cudaMemcpyKind kind, int ncomp = 6) {
    const size_t w = (size_t)h->V * elem;
    const size_t dp = (dst_padded ? (size_t)h->cs : (size_t)h->V) * elem;
    const size_t sp = (src_padded ? (size_t)h->cs : (size_t)h->V) * elem;
    return cudaMemcpy2DAsync(dst, dp, src, sp, w, ncomp, kind, h->stream);
}

static inline double* cell_field(double* base, const fftg_handle* h, int c) {
    return base + (size_t)c * 6 * h->cs;
}

// Constitutive update of `ncells` cells starting at cell0 at E (Edev, one
// 6-vector per cell) + eps against the committed history; mask_dev (may be
// null) skips cells.
static int launch_constitutive(fftg_handle* h, const int* mask_dev, int ncells, int cell0,
                               const double* eps, double* sigma, bool write_history, CGState* cg,
                               bool write_tangent = true, bool elastic_only = false) {
    ConstArgs a{};
    a.V = h->V;
    a.cs = h->cs;
    a.Edev = h->Edev + 6 * cell0;
    a.eps = eps + (size_t)cell0 * 6 * h->cs;
    a.eps_p = h->eps_p + (size_t)cell0 * 6 * h->cs;
    a.epbar = h->epbar + (size_t)cell0 * h->cs;
    a.phase = h->phase + (size_t)cell0 * h->cs;
    a.mats = h->mats;
    a.sigma = sigma ? sigma + (size_t)cell0 * 6 * h->cs : nullptr;
    a.eps_p_new = write_history ? h->eps_p_tr + (size_t)cell0 * 6 * h->cs : nullptr;
    a.epbar_new = write_history ? h->epbar_tr + (size_t)cell0 * h->cs : nullptr;
    a.tangent = write_tangent ? (char*)h->tangent + (size_t)cell0 * 7 * h->cs * (h->mixed ? 4 : 8)
                              : nullptr;
    a.partials = h->partials;
    a.nd = h->nd + cell0;
    a.cg = cg ? cg + cell0 : nullptr;
    a.tie = 1e-12;
    a.dt = h->opt.dt;
    a.elastic_only = elastic_only ? 1 : 0;
    a.skip_sums = write_history ? 0 : 1;  // Sigma is read after the commit's call only
    a.active = mask_dev ? mask_dev + cell0 : nullptr;
    a.cell_fields = 6 * h->cs;
    a.cell_scalar = h->cs;
    a.cell_tangent = 7 * h->cs;
    const dim3 g(pointwise_blocks(h->V), ncells);
    const int slot = prof_begin(h, h->mixed ? KK_CONSTITUTIVE_F32 : KK_CONSTITUTIVE_F64);
    if (h->mixed)
        k_constitutive<float><<<g, kThreads, 0, h->stream>>>(a);
    else
        k_constitutive<double><<<g, kThreads, 0, h->stream>>>(a);
    prof_end(h, slot);
    CK(cudaGetLastError());
    if (write_tangent)
        for (int b = cell0; b < cell0 + ncells; ++b)
            if (!mask_dev || (mask_dev == h->active && h->h_active[b])) h->have_update[b] = 1;
    return FFTG_OK;
}

// Forward-project-inverse core on the spectrum buffer (P2, P3, P4).
static PassArgs base_args_fft(fftg_handle* h, int prec) {
    PassArgs a = base_args(h, prec != FFT_F32);
    if (prec == FFT_DD) a.tw = h->twdd;
    return a;
}

static int run_p234(fftg_handle* h, int prec, double scale, CGState* cg, int nf, const int* mask,
                    const double* red_in = nullptr, int red_n = 0) {
    PassArgs a = base_args_fft(h, prec);
    a.out = h->spec;
    a.cg = cg;
    a.scale = scale;
    a.active = mask;
    a.red_in = red_in;
    a.red_n = red_n;
    const PassKind k2 = prec == FFT_DD ? PK_P2_DD : prec == FFT_F64 ? PK_P2_F64 : PK_P2_F32;
    const PassKind k3 = prec == FFT_DD ? PK_P3_DD : prec == FFT_F64 ? PK_P3_F64 : PK_P3_F32;
    const PassKind k4 = prec == FFT_DD ? PK_P4_DD : prec == FFT_F64 ? PK_P4_F64 : PK_P4_F32;
    CK(pass(h, k2, a, nf));
    a.red_in = nullptr;
    CK(pass(h, k3, a, nf));
    CK(pass(h, k4, a, nf));
    return FFTG_OK;
}

// r = -G sigma for the cells in the active mask (FP64 FFTs, or double-float
// ones in the mixed path), rounded to the inner precision; x = 0.
static int launch_residual(fftg_handle* h) {
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    const bool dd = h->mixed && FFTG_RESIDUAL_DD;
    PassArgs a = base_args_fft(h, dd ? FFT_DD : FFT_F64);
    a.in = h->sigma;
    a.out = h->spec;
    a.active = h->active;
    CK(pass(h, dd ? PK_P1_PLAIN_DD : PK_P1_PLAIN_F64, a, h->B));
    int rc = run_p234(h, dd ? FFT_DD : FFT_F64, -invN3, nullptr, h->B, h->active);
    if (rc) return rc;
    PassArgs b = base_args_fft(h, dd ? FFT_DD : FFT_F64);
    b.in = h->spec;
    b.out = h->r;
    b.cg = h->cg;
    b.active = h->active;
    CK(pass(h, dd ? PK_P5_RHS_DD_TO_F32 : h->mixed ? PK_P5_RHS_F64_TO_F32 : PK_P5_RHS_F64_TO_F64, b, h->B));
    CK(cudaMemsetAsync(h->x, 0, (size_t)h->B * 6 * h->cs * (h->mixed ? 4 : 8), h->stream));
    return FFTG_OK;
}

// The mixed path's CG (not the basic scheme) runs without the update pass:
// alpha from <p, C : p> in P1, r -= alpha q in P5 (passes.cuh, P1_CGF).
// 0: P1_CG / P5_DOT and the update pass, as in the FP64 path.
#ifndef FFTG_CG_FUSED
#define FFTG_CG_FUSED 1
#endif
static bool cg_fused(const fftg_handle* h) {
    return FFTG_CG_FUSED && h->mixed && h->opt.solver == FFTG_SOLVER_CG;
}

// One CG iteration on nf fields: the fused matvec passes and the update.
// `tangent`/`tstride`: per-field tangents (batched cells) or one shared.
static int launch_cg_iteration(fftg_handle* h, int nf, const void* tangent, long long tstride) {
    const bool f64 = !h->mixed;
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    if (cg_fused(h)) {
        PassArgs a = base_args(h, false);
        a.aux = h->r;
        a.aux2 = h->p;
        a.aux3 = h->x;
        a.tangent = tangent;
        a.tstride = tstride;
        a.out = h->spec;
        a.cg = h->cg;
        CK(pass(h, PK_P1_CGF_F32, a, nf));
        // P2 reduces P1's block partials of <p, C : p> (alpha)
        const int nb1 = variant_shape(h->N, TK_P1, schedule_variant(h->N, TK_P1)).blocks;
        int rc = run_p234(h, FFT_F32, invN3, h->cg, nf, nullptr, h->partials, nb1);
        if (rc) return rc;
        PassArgs b = base_args(h, false);
        b.in = h->spec;
        b.aux = h->r;
        b.aux3 = h->r;
        b.cg = h->cg;
        CK(pass(h, PK_P5_CGF_F32, b, nf));
        // <r, r> from P5's block partials: beta and the stopping tests
        const int nb5 = variant_shape(h->N, TK_P5, schedule_variant(h->N, TK_P5)).blocks;
        const int slot = prof_begin(h, KK_CG_RR);
        k_cg_rr<<<nf, 1024, 0, h->stream>>>(h->partials, nb5, h->cg);
        prof_end(h, slot);
        CK(cudaGetLastError());
        return FFTG_OK;
    }
    PassArgs a = base_args(h, f64);
    a.aux = h->r;
    a.aux2 = h->p;
    a.aux3 = h->x;
    a.tangent = tangent;
    a.tstride = tstride;
    a.out = h->spec;
    a.cg = h->cg;
    CK(pass(h, f64 ? PK_P1_CG_F64 : PK_P1_CG_F32, a, nf));
    int rc = run_p234(h, f64 ? FFT_F64 : FFT_F32, invN3, h->cg, nf, nullptr);
    if (rc) return rc;
    PassArgs b = base_args(h, f64);
    b.in = h->spec;
    b.out = h->q;
    b.aux = h->p;
    b.cg = h->cg;
    CK(pass(h, f64 ? PK_P5_DOT_F64 : PK_P5_DOT_F32, b, nf));
    VecArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.x = h->x;
    u.r = h->r;
    u.p = h->p;
    u.q = h->q;
    u.cg = h->cg;
    u.partials = h->partials;
    u.fstride = 6 * h->cs;
    dim3 g(vector_blocks(h->cs, f64 ? 8 : 4), 1, nf);
    const int slot = prof_begin(h, f64 ? KK_CG_UPDATE_F64 : KK_CG_UPDATE_F32);
    if (f64)
        k_cg_update<double><<<g, kThreads, 0, h->stream>>>(u);
    else
        k_cg_update<float><<<g, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

namespace fftg {
// Loop condition of the device-resident CG (a conditional WHILE node of a
// CUDA graph): go on while any of the nf solves is running. `guard` counts
// the passes of the loop body; past `cap` passes the loop stops whatever the
// solves report, so the loop always ends.
__global__ void k_cg_continue(cudaGraphConditionalHandle cond, const CGState* cg, int nf,
                              unsigned int* guard, unsigned int cap) {
    if (threadIdx.x != 0) return;
    bool any = false;
    for (int f = 0; f < nf; ++f) any = any || (cg[f].done == CG_RUNNING);
    const unsigned int n = ++(*guard);
    if (n >= cap) any = false;
    cudaGraphSetConditional(cond, any ? 1u : 0u);
}

}  // namespace fftg

// Device-resident CG: one graph whose conditional WHILE node repeats the
// iteration (the five passes and the update) while any solve is running;
// k_cg_continue sets the condition on the device, so the host launches the
// whole solve once and waits once.
static int build_cg_graph(fftg_handle* h, int nf, const void* tangent, long long tstride,
                          fftg_handle::CgGraph* g) {
    g->nf = nf;
    g->tangent = tangent;
    g->tstride = tstride;
    if (cudaGraphCreate(&g->graph, 0) != cudaSuccess) return FFTG_ECUDA;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, g->graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return FFTG_ECUDA;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g->graph, nullptr, nullptr, 0, &p) != cudaSuccess) return FFTG_ECUDA;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess)
        return FFTG_ECUDA;
    int rc = launch_cg_iteration(h, nf, tangent, tstride);
    const unsigned int cap =
        (unsigned int)((h->opt.fixed_cg > 0 ? h->opt.fixed_cg : h->opt.max_cg) + 4);
    if (rc == FFTG_OK) {
        k_cg_continue<<<1, 32, 0, h->stream>>>(cond, h->cg, nf, h->guard, cap);
        if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
    }
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(h->stream, &captured) != cudaSuccess || rc) return FFTG_ECUDA;
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) return FFTG_ECUDA;
    return FFTG_OK;
}

static void free_graphs(fftg_handle* h) {
    for (auto& g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    h->graphs.clear();
}

// The cached graph for (nf, tangent, tstride), built on first use (at most
// four are kept; the least recently used is rebuilt on demand).
static fftg_handle::CgGraph* cg_graph_for(fftg_handle* h, int nf, const void* tangent, long long tstride) {
    for (auto& g : h->graphs)
        if (g.nf == nf && g.tangent == tangent && g.tstride == tstride) {
            g.used = ++h->graph_clock;
            return &g;
        }
    if (h->graphs.size() >= 4) {
        auto lru = std::min_element(h->graphs.begin(), h->graphs.end(),
                                    [](const auto& a, const auto& b) { return a.used < b.used; });
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        if (lru->graph) cudaGraphDestroy(lru->graph);
        h->graphs.erase(lru);
    }
    fftg_handle::CgGraph g;
    const long long launches_before = h->launches;
    if (build_cg_graph(h, nf, tangent, tstride, &g) != FFTG_OK) {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(h->stream, &junk);
            if (junk) cudaGraphDestroy(junk);
        }
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        cudaGetLastError();
        h->launches = launches_before;
        return nullptr;
    }
    h->launches = launches_before;  // capture enqueued nothing
    g.used = ++h->graph_clock;
    h->graphs.push_back(g);
    return &h->graphs.back();
}

// Mixed precision: x <- G x (FP32 passes) on the nf solution fields. The
// FP32 recursion of CG lets the residual, and with it x, drift out of the
// compatible space (by about 1e-5 of |x| over some tens of iterations:
// each q = G (C : p) carries FP32 rounding). Newton's corrections then add
// an incompatible part to eps* that no later correction removes, and the
// converged state sits off the FP64 solution by that much. One projection
// per solve brings the incompatible part down to the rounding of a single
// FP32 projection.
#ifndef FFTG_PROJECT_X
#define FFTG_PROJECT_X 1
#endif
static int project_solution(fftg_handle* h, int nf, const int* active) {
    if (!h->mixed || !FFTG_PROJECT_X) return FFTG_OK;
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    PassArgs a = base_args(h, false);
    a.in = h->x;
    a.out = h->spec;
    a.active = active;
    CK(pass(h, PK_P1_PLAIN_F32, a, nf));
    int rc = run_p234(h, FFT_F32, invN3, nullptr, nf, active);
    if (rc) return rc;
    PassArgs b = base_args(h, false);
    b.in = h->spec;
    b.out = h->x;
    b.active = active;
    CK(pass(h, PK_P5_PLAIN_F32, b, nf));
    return FFTG_OK;
}

// Basic scheme: the Richardson step of each of the nf CG states from the
// extreme eigenvalues of the tangent(s), after the right-hand side pass.
// ncells cells with nw states each (Newton: B cells x 1; tangent: 1 x 6).
static int launch_bounds(fftg_handle* h, const void* tangent, long long cell_tangent, int ncells, int nw,
                         const int* active) {
    if (h->opt.solver != FFTG_SOLVER_RICHARDSON) return FFTG_OK;
    VecArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.tangent = tangent;
    u.cell_tangent = cell_tangent;
    u.nw = nw;
    u.cg = h->cg;
    u.nd = h->nd;
    u.partials = h->partials;
    u.active = active;
    const dim3 g(pointwise_blocks(h->V), ncells);
    const int slot = prof_begin(h, KK_TANGENT_BOUNDS);
    if (h->mixed)
        k_tangent_bounds<float><<<g, kThreads, 0, h->stream>>>(u);
    else
        k_tangent_bounds<double><<<g, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

// x += alpha p for the solves whose last update left that step pending.
static int launch_cg_finish(fftg_handle* h, int nf) {
    const bool f64 = !h->mixed;
    VecArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.x = h->x;
    u.p = h->p;
    u.cg = h->cg;
    u.fstride = 6 * h->cs;
    dim3 g(vector_blocks(6 * h->cs, f64 ? 8 : 4), 1, nf);
    const int slot = prof_begin(h, f64 ? KK_CG_FINISH_F64 : KK_CG_FINISH_F32);
    if (f64)
        k_cg_finish<double><<<g, kThreads, 0, h->stream>>>(u);
    else
        k_cg_finish<float><<<g, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

// Runs CG iterations until every one of the nf solves is done: as one graph
// launch (device-resident loop), or, with profiling on or graphs disabled,
// in chunks enqueued from the host (kernels of a finished solve return at
// entry, so a chunk may overrun the last iteration without effect).
static int run_cg(fftg_handle* h, int nf, const void* tangent, long long tstride) {
    const bool profiling = h->prof && h->prof->on;
    if (h->opt.cg_graph && !profiling && !h->graphs_broken) {
        fftg_handle::CgGraph* g = cg_graph_for(h, nf, tangent, tstride);
        if (g) {
            CK(cudaMemsetAsync(h->guard, 0, sizeof(unsigned int), h->stream));
            CK(cudaGraphLaunch(g->exec, h->stream));
            int rc = launch_cg_finish(h, nf);
            if (rc) return rc;
            // one launch of each kernel of an iteration per loop pass
            CK(cudaMemcpyAsync(h->h_cg, h->cg, nf * sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            int maxit = 0;
            for (int f = 0; f < nf; ++f) maxit = std::max(maxit, h->h_cg[f].it);
            h->launches += 7LL * (maxit + 1);
            return FFTG_OK;
        }
        h->graphs_broken = true;
    }
    CK(cudaMemcpyAsync(h->h_cg, h->cg, nf * sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int chunk = 2;
    int launched = 0;
    const int cap = (h->opt.fixed_cg > 0 ? h->opt.fixed_cg : h->opt.max_cg) + 1;
    for (;;) {
        bool all = true;
        for (int f = 0; f < nf; ++f) all = all && h->h_cg[f].done != CG_RUNNING;
        if (all) break;
        if (launched > cap) return FFTG_ENOCONV_CG;  // defensive: should not happen
        for (int k = 0; k < chunk; ++k) {
            int rc = launch_cg_iteration(h, nf, tangent, tstride);
            if (rc) return rc;
        }
        launched += chunk;
        chunk = std::min(chunk * 2, 16);
        CK(cudaMemcpyAsync(h->h_cg, h->cg, nf * sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return launch_cg_finish(h, nf);
}

static void set_cg_params(fftg_handle* h, int nf, double tol, const int* run) {
    for (int f = 0; f < h->nf; ++f) {
        CGState& c = h->h_cg[f];
        std::memset(&c, 0, sizeof(CGState));
        c.tol2 = tol * tol;
        c.max_it = h->opt.max_cg;
        c.fixed_it = h->opt.fixed_cg;
        // the FP32 inner solve stops when it stagnates (FP64 Newton refines)
        c.stag_window = (h->mixed && h->opt.fixed_cg <= 0) ? kStagWindow : 0;
        const bool on = f < nf && (!run || run[f]);
        c.done = on ? CG_RUNNING : CG_CONVERGED;
    }
}

// eps* += d eps for the cells in the active mask, with ||d eps||^2 per cell
// (Algorithm 1, iterative update).
static int launch_newton_update(fftg_handle* h) {
    VecArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.x = h->x;
    u.eps = h->eps_work;
    u.nd = h->nd;
    u.partials = h->partials;
    u.active = h->active;
    u.fstride = 6 * h->cs;
    u.cell_fields = 6 * h->cs;
    const dim3 g(pointwise_blocks(h->V), h->B);
    const int slot = prof_begin(h, h->mixed ? KK_NEWTON_UPDATE_F32 : KK_NEWTON_UPDATE_F64);
    if (h->mixed)
        k_newton_update<float><<<g, kThreads, 0, h->stream>>>(u);
    else
        k_newton_update<double><<<g, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    return FFTG_OK;
}

// ---------------------------------------------------------------- Newton rounds
namespace fftg_detail {

int newton_round(fftg_handle* h, const int* run, double tol_inner, RoundOut* out) {
    const int B = h->B;
    for (int b = 0; b < B; ++b) h->h_active[b] = run[b];
    CK(cudaMemcpyAsync(h->active, h->h_active, B * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    set_cg_params(h, B, tol_inner, run);
    CK(cudaMemcpyAsync(h->cg, h->h_cg, h->nf * sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
    int rc = launch_constitutive(h, h->active, B, 0, h->eps_work, h->sigma, false, h->cg);
    if (rc) return rc;
    rc = launch_residual(h);
    if (rc) return rc;
    rc = launch_bounds(h, h->tangent, 7 * h->cs, B, 1, h->active);
    if (rc) return rc;
    rc = run_cg(h, B, h->tangent, 7 * h->cs);
    if (rc) return rc;
    rc = project_solution(h, B, h->active);
    if (rc) return rc;
    rc = launch_newton_update(h);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->h_cg, h->cg, B * sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->h_nd, h->nd, B * sizeof(NewtonDev), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int b = 0; b < B; ++b) {
        if (!run[b]) continue;
        const CGState& c = h->h_cg[b];
        out[b].cg_it = c.it;
        out[b].cg_done = c.done;
        out[b].de2 = h->h_nd[b].de2;
        out[b].gs2 = c.gs2;
        out[b].sig2 = h->h_nd[b].sig2;
        out[b].relres = c.rr0 > 0 ? std::sqrt(c.rr / c.rr0) : 0.0;
    }
    return FFTG_OK;
}

int set_trial_strain(fftg_handle* h, int cell, const double Et[6], bool copy_eps) {
    std::memcpy(h->h_E + 6 * cell, Et, 6 * sizeof(double));
    CK(cudaMemcpyAsync(h->Edev + 6 * cell, h->h_E + 6 * cell, 6 * sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    if (copy_eps)
        CK(cudaMemcpyAsync(cell_field(h->eps_work, h, cell), cell_field(h->eps_star, h, cell),
                           6 * h->cs * 8, cudaMemcpyDeviceToDevice, h->stream));
    return FFTG_OK;
}

// Final constitutive call of the cells in `fin` (history out), their
// homogenised stress, and the commit of their trial state.
int finish_cells(fftg_handle* h, const int* fin, double* sigma_out) {
    const int B = h->B;
    for (int b = 0; b < B; ++b) h->h_active[b] = fin[b];
    CK(cudaMemcpyAsync(h->active, h->h_active, B * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    int rc = launch_constitutive(h, h->active, B, 0, h->eps_work, h->sigma, true, nullptr);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->h_nd, h->nd, B * sizeof(NewtonDev), cudaMemcpyDeviceToHost, h->stream));
    int all = 1;
    for (int b = 0; b < B; ++b) all &= fin[b];
    if (all) {
        CK(cudaMemcpyAsync(h->eps_star, h->eps_work, (size_t)B * 6 * h->cs * 8, cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(cudaMemcpyAsync(h->eps_p, h->eps_p_tr, (size_t)B * 6 * h->cs * 8, cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(cudaMemcpyAsync(h->epbar, h->epbar_tr, (size_t)B * h->cs * 8, cudaMemcpyDeviceToDevice,
                           h->stream));
    } else {
        for (int b = 0; b < B; ++b) {
            if (!fin[b]) continue;
            CK(cudaMemcpyAsync(cell_field(h->eps_star, h, b), cell_field(h->eps_work, h, b), 6 * h->cs * 8,
                               cudaMemcpyDeviceToDevice, h->stream));
            CK(cudaMemcpyAsync(cell_field(h->eps_p, h, b), cell_field(h->eps_p_tr, h, b), 6 * h->cs * 8,
                               cudaMemcpyDeviceToDevice, h->stream));
            CK(cudaMemcpyAsync(h->epbar + (size_t)b * h->cs, h->epbar_tr + (size_t)b * h->cs, h->cs * 8,
                               cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    for (int b = 0; b < B; ++b) {
        if (!fin[b]) continue;
        for (int c = 0; c < 6; ++c) {
            sigma_out[6 * b + c] = h->h_nd[b].sum[c] / (double)h->V;
            h->E[6 * b + c] = h->h_E[6 * b + c];
        }
        h->have_tangent[b] = 1;
    }
    return FFTG_OK;
}

int cells(const fftg_handle* h) { return h->B; }
int grid_n(const fftg_handle* h) { return h->N; }
bool is_mixed(const fftg_handle* h) { return h->mixed != 0; }
const fftg_options& options(const fftg_handle* h) { return h->opt; }
const double* committed_E(const fftg_handle* h, int cell) { return h->E.data() + 6 * cell; }
long long voxels(const fftg_handle* h) { return h->V; }

int upload_cell(fftg_handle* h, int cell, const uint8_t* phase, const double* state) {
    if (phase)
        CK(cudaMemcpyAsync(h->phase + (size_t)cell * h->cs, phase, h->V, cudaMemcpyHostToDevice, h->stream));
    if (state) {
        const double* d = state;
        CK(copy_field(h, cell_field(h->eps_star, h, cell), true, d + 6, false, 8, cudaMemcpyHostToDevice));
        CK(copy_field(h, cell_field(h->eps_p, h, cell), true, d + 6 + 6 * h->V, false, 8,
                      cudaMemcpyHostToDevice));
        CK(cudaMemcpyAsync(h->epbar + (size_t)cell * h->cs, d + 6 + 12 * h->V, h->V * 8,
                           cudaMemcpyHostToDevice, h->stream));
        std::memcpy(h->E.data() + 6 * cell, d, 6 * sizeof(double));
    } else {
        CK(cudaMemsetAsync(cell_field(h->eps_star, h, cell), 0, 6 * h->cs * 8, h->stream));
        CK(cudaMemsetAsync(cell_field(h->eps_p, h, cell), 0, 6 * h->cs * 8, h->stream));
        CK(cudaMemsetAsync(h->epbar + (size_t)cell * h->cs, 0, h->cs * 8, h->stream));
        std::fill(h->E.begin() + 6 * cell, h->E.begin() + 6 * cell + 6, 0.0);
    }
    h->have_tangent[cell] = 0;
    h->have_update[cell] = 0;
    CK(cudaStreamSynchronize(h->stream));
    return FFTG_OK;
}

int download_cell(fftg_handle* h, int cell, double* state) {
    double* d = state;
    std::memcpy(d, h->E.data() + 6 * cell, 6 * sizeof(double));
    CK(copy_field(h, d + 6, false, cell_field(h->eps_star, h, cell), true, 8, cudaMemcpyDeviceToHost));
    CK(copy_field(h, d + 6 + 6 * h->V, false, cell_field(h->eps_p, h, cell), true, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpyAsync(d + 6 + 12 * h->V, h->epbar + (size_t)cell * h->cs, h->V * 8, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FFTG_OK;
}

// Newton test of one cell after a round (Algorithm 1): returns 0 while the
// cell keeps iterating, 1 when it has converged, or an FFTG_E* code.
int newton_decide(fftg_handle* h, int cell, const RoundOut& ro, double normE, double tol_newton, int* it) {
    fftg_stats& st = h->stats[cell];
    const double nde = std::sqrt(ro.de2);
    const double rel = normE > 0 ? nde / normE : (nde == 0 ? 0.0 : INFINITY);
    const int i = *it;
    if (i < FFTG_MAX_NEWTON_LOG) {
        st.cg_per_newton[i] = ro.cg_it;
        st.newton_norm[i] = rel;
        st.residual[i] = ro.sig2 > 0 ? std::sqrt(ro.gs2 / ro.sig2) : 0.0;
        st.cg_relres[i] = ro.relres;
        st.cg_status[i] = ro.cg_done;
    }
    st.cg_iters += ro.cg_it;
    *it = i + 1;
    st.newton_iters = *it;
    if (ro.cg_done == CG_BREAKDOWN || !std::isfinite(rel)) return FFTG_ENAN;
    if (h->opt.fixed_newton > 0) return *it >= h->opt.fixed_newton ? 1 : 0;
    if (rel <= tol_newton || nde == 0.0) return 1;
    if (*it >= h->opt.max_newton) return FFTG_ENOCONV_NEWTON;
    return 0;
}

void reset_stats(fftg_handle* h, int cell) {
    std::memset(&h->stats[cell], 0, sizeof(fftg_stats));
    h->have_tangent[cell] = 0;
}

void set_status(fftg_handle* h, int cell, int status) { h->stats[cell].status = status; }

}  // namespace fftg_detail

using namespace fftg_detail;

// One increment for every cell (Algorithm 1, increment loop body), cells in
// lock step but each with its own Newton test.
static int batch_step(fftg_handle* h, const double* dE, double tol_newton, double tol_cg, double* sigma_out,
                      int* newton_iters, int* cg_iters, int* status) {
    const int B = h->B;
    const double tol_inner = h->mixed ? std::max(tol_cg, h->opt.cg_inner_floor) : tol_cg;
    std::vector<double> normE(B);
    std::vector<int> run(B, 1), fin(B, 0), it(B, 0);
    for (int b = 0; b < B; ++b) {
        double Et[6];
        for (int c = 0; c < 6; ++c) Et[c] = h->E[6 * b + c] + dE[6 * b + c];
        normE[b] = std::sqrt((double)h->V) * frob6(Et);
        std::memcpy(h->h_E + 6 * b, Et, sizeof(Et));
        reset_stats(h, b);
        status[b] = FFTG_OK;
    }
    CK(cudaMemcpyAsync(h->Edev, h->h_E, (size_t)B * 6 * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->eps_work, h->eps_star, (size_t)B * 6 * h->cs * 8, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<RoundOut> ro(B);
    for (;;) {
        bool any = false;
        for (int b = 0; b < B; ++b) any = any || run[b];
        if (!any) break;
        int rc = newton_round(h, run.data(), tol_inner, ro.data());
        if (rc) return rc;
        for (int b = 0; b < B; ++b) {
            if (!run[b]) continue;
            const int d = newton_decide(h, b, ro[b], normE[b], tol_newton, &it[b]);
            if (d == 1) {
                run[b] = 0;
                fin[b] = 1;
            } else if (d < 0) {
                status[b] = d;
                run[b] = 0;
            }
        }
    }
    bool anyfin = false;
    for (int b = 0; b < B; ++b) anyfin = anyfin || fin[b];
    if (anyfin) {
        int rc = finish_cells(h, fin.data(), sigma_out);
        if (rc) return rc;
    }
    int first = FFTG_OK;
    for (int b = 0; b < B; ++b) {
        h->stats[b].status = status[b];
        if (newton_iters) newton_iters[b] = it[b];
        if (cg_iters) cg_iters[b] = h->stats[b].cg_iters;
        if (status[b] != FFTG_OK && first == FFTG_OK) first = status[b];
    }
    return first;
}

// ---------------------------------------------------------------- device-driven increments
// A group of batch handles (cells of several grid sizes) whose increment
// runs as one CUDA graph launch: per handle, a branch with no dependency on
// the others, holding
//   k_inc_begin, eps_work <- eps*,
//   WHILE (a cell of the handle iterates Newton):           [device test]
//     k_inc_cg_reset, stress update, residual G sigma, [bounds],
//     WHILE (a CG solve runs): one CG iteration              [device test]
//     pending CG step, projection of the inner solution, eps* += d eps,
//     k_inc_decide (Newton test of Algorithm 1, sets the outer condition)
//   commit: stress update with history, homogenised stress, trial ->
//   committed state of the converged cells.
// The branches of different grid sizes run concurrently on the device.
struct fftg_group {
    std::vector<fftg_handle*> hs;
    std::vector<cudaStream_t> cap;      // two capture streams per handle
    cudaStream_t stream = nullptr;      // the graph's launch stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double tol_newton = -1.0, tol_cg = -1.0;
    std::vector<std::vector<IncDev>> h_inc;
    long long launches = 0;
};

namespace {

// Adds a WHILE node after the work captured so far on `s` (a stream capturing
// into some graph) and returns its body; the capture continues after it.
int add_while(cudaStream_t s, cudaGraphConditionalHandle cond, cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edges, &ndeps) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return FFTG_ECUDA;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, edges, ndeps, &p) != cudaSuccess) return FFTG_ECUDA;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return FFTG_ECUDA;
    *body = p.conditional.phGraph_out[0];
    return FFTG_OK;
}

IncArgs inc_args(fftg_handle* h, double tol_newton, double tol_inner) {
    IncArgs a{};
    a.B = h->B;
    a.V = h->V;
    a.run = h->run_dev;
    a.dE = h->dE_dev;
    a.Ecom = h->Ecom_dev;
    a.Etrial = h->Edev;
    a.active = h->active;
    a.fin = h->fin_dev;
    a.inc = h->inc_dev;
    a.cg = h->cg;
    a.nd = h->nd;
    a.tol_newton = tol_newton;
    a.max_newton = h->opt.max_newton;
    a.fixed_newton = h->opt.fixed_newton;
    a.newton_guard = h->guard + 1;
    a.cg_guard = h->guard;
    a.newton_cap = (unsigned int)((h->opt.fixed_newton > 0 ? h->opt.fixed_newton : h->opt.max_newton) + 2);
    CGState& c = a.cg_template;
    c.tol2 = tol_inner * tol_inner;
    c.max_it = h->opt.max_cg;
    c.fixed_it = h->opt.fixed_cg;
    c.stag_window = (h->mixed && h->opt.fixed_cg <= 0) ? kStagWindow : 0;
    return a;
}

// One handle's branch of the group graph, captured on s1 (into the graph it
// is capturing) with the Newton body on s2 and the CG body on s3.
int capture_branch(fftg_handle* h, cudaGraph_t top, cudaStream_t s1, cudaStream_t s2, cudaStream_t s3,
                   double tol_newton, double tol_cg) {
    const double tol_inner = h->mixed ? std::max(tol_cg, h->opt.cg_inner_floor) : tol_cg;
    IncArgs ia = inc_args(h, tol_newton, tol_inner);
    cudaStream_t own = h->stream;
    int rc = FFTG_OK;
    cudaGraphConditionalHandle cN, cC;
    cudaGraph_t bodyN = nullptr, bodyC = nullptr;
    h->stream = s1;
    if (cudaStreamBeginCaptureToGraph(s1, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        h->stream = own;
        return FFTG_ECUDA;
    }
    if (cudaGraphConditionalHandleCreate(&cN, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        rc = FFTG_ECUDA;
    } else {
        k_inc_begin<<<1, kThreads, 0, s1>>>(cN, ia);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h->eps_work, h->eps_star, (size_t)h->B * 6 * h->cs * 8, cudaMemcpyDeviceToDevice,
                            s1) != cudaSuccess)
            rc = FFTG_ECUDA;
    }
    if (rc == FFTG_OK) rc = add_while(s1, cN, &bodyN);
    // the Newton body
    if (rc == FFTG_OK) {
        h->stream = s2;
        if (cudaStreamBeginCaptureToGraph(s2, bodyN, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess) {
            rc = FFTG_ECUDA;
        } else {
            if (cudaGraphConditionalHandleCreate(&cC, bodyN, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
                rc = FFTG_ECUDA;
            } else {
                k_inc_cg_reset<<<1, kThreads, 0, s2>>>(cC, ia);
                if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
            }
            if (rc == FFTG_OK) rc = launch_constitutive(h, h->active, h->B, 0, h->eps_work, h->sigma, false, h->cg);
            if (rc == FFTG_OK) rc = launch_residual(h);
            if (rc == FFTG_OK) rc = launch_bounds(h, h->tangent, 7 * h->cs, h->B, 1, h->active);
            if (rc == FFTG_OK) rc = add_while(s2, cC, &bodyC);
            // the CG body
            if (rc == FFTG_OK) {
                h->stream = s3;
                if (cudaStreamBeginCaptureToGraph(s3, bodyC, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
                    cudaSuccess) {
                    rc = FFTG_ECUDA;
                } else {
                    rc = launch_cg_iteration(h, h->B, h->tangent, 7 * h->cs);
                    const unsigned int cap =
                        (unsigned int)((h->opt.fixed_cg > 0 ? h->opt.fixed_cg : h->opt.max_cg) + 4);
                    if (rc == FFTG_OK) {
                        k_cg_continue<<<1, 32, 0, s3>>>(cC, h->cg, h->B, h->guard, cap);
                        if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
                    }
                    cudaGraph_t g3 = nullptr;
                    if (cudaStreamEndCapture(s3, &g3) != cudaSuccess) rc = FFTG_ECUDA;
                }
                h->stream = s2;
            }
            if (rc == FFTG_OK) rc = launch_cg_finish(h, h->B);
            if (rc == FFTG_OK) rc = project_solution(h, h->B, h->active);
            if (rc == FFTG_OK) rc = launch_newton_update(h);
            if (rc == FFTG_OK) {
                k_inc_decide<<<1, kThreads, 0, s2>>>(cN, ia);
                if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
            }
            cudaGraph_t g2 = nullptr;
            if (cudaStreamEndCapture(s2, &g2) != cudaSuccess) rc = FFTG_ECUDA;
        }
        h->stream = s1;
    }
    // the commit of the converged cells
    if (rc == FFTG_OK) rc = launch_constitutive(h, h->fin_dev, h->B, 0, h->eps_work, h->sigma, true, nullptr);
    if (rc == FFTG_OK) {
        k_inc_end<<<1, kThreads, 0, s1>>>(ia);
        CommitArgs ca{};
        ca.fin = h->fin_dev;
        ca.eps_star = h->eps_star;
        ca.eps_work = h->eps_work;
        ca.eps_p = h->eps_p;
        ca.eps_p_tr = h->eps_p_tr;
        ca.epbar = h->epbar;
        ca.epbar_tr = h->epbar_tr;
        ca.cs = h->cs;
        k_inc_commit<<<dim3(vector_blocks(6 * h->cs, 8), h->B), kThreads, 0, s1>>>(ca);
        if (cudaGetLastError() != cudaSuccess) rc = FFTG_ECUDA;
    }
    cudaGraph_t g1 = nullptr;
    if (cudaStreamEndCapture(s1, &g1) != cudaSuccess) rc = FFTG_ECUDA;
    h->stream = own;
    return rc;
}

void group_free_graph(fftg_group* g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
}

int group_build(fftg_group* g, double tol_newton, double tol_cg) {
    group_free_graph(g);
    if (cudaGraphCreate(&g->graph, 0) != cudaSuccess) return FFTG_ECUDA;
    int rc = FFTG_OK;
    for (size_t k = 0; k < g->hs.size() && rc == FFTG_OK; ++k) {
        fftg_handle* h = g->hs[k];
        const long long before = h->launches;
        const bool prof_on = h->prof && h->prof->on;
        if (prof_on) h->prof->on = false;  // no per-launch events inside the graph
        rc = capture_branch(h, g->graph, g->cap[3 * k], g->cap[3 * k + 1], g->cap[3 * k + 2], tol_newton, tol_cg);
        if (prof_on) h->prof->on = true;
        h->launches = before;  // capture enqueues nothing
    }
    if (rc == FFTG_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = FFTG_ECUDA;
    if (rc != FFTG_OK) {
        cudaGetLastError();
        group_free_graph(g);
        return rc;
    }
    g->tol_newton = tol_newton;
    g->tol_cg = tol_cg;
    return FFTG_OK;
}

}  // namespace

// ---------------------------------------------------------------- public API
extern "C" {

int fftg_group_create(fftg_group** out, fftg_handle* const* handles, int n) {
    if (!out || !handles || n < 1) return FFTG_EINVAL;
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!handles[k] || handles[k]->opt.solver != FFTG_SOLVER_CG) return FFTG_EINVAL;
        for (int j = 0; j < k; ++j)
            if (handles[j] == handles[k]) return FFTG_EINVAL;
    }
    fftg_group* g = new (std::nothrow) fftg_group();
    if (!g) return FFTG_ENOMEM;
    g->hs.assign(handles, handles + n);
    g->h_inc.resize(n);
    bool ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess;
    g->cap.assign(3 * n, nullptr);
    for (int k = 0; k < 3 * n && ok; ++k) ok = cudaStreamCreateWithFlags(&g->cap[k], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < n; ++k) g->h_inc[k].resize(handles[k]->B);
    if (!ok) {
        cudaGetLastError();
        fftg_group_destroy(g);
        return FFTG_ECUDA;
    }
    *out = g;
    return FFTG_OK;
}

void fftg_group_destroy(fftg_group* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    group_free_graph(g);
    for (cudaStream_t s : g->cap)
        if (s) cudaStreamDestroy(s);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

int fftg_group_step(fftg_group* g, const double* dE, const int* run, double tol_newton, double tol_cg,
                    double* sigma_out, int* newton_iters, int* cg_iters, int* status) {
    if (!g || !dE || !sigma_out || !status || !(tol_newton > 0) || !(tol_cg > 0)) return FFTG_EINVAL;
    size_t total = 0;
    for (fftg_handle* h : g->hs) total += (size_t)h->B;
    for (size_t i = 0; i < 6 * total; ++i)
        if (!std::isfinite(dE[i])) return FFTG_ENAN;
    for (fftg_handle* h : g->hs)
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FFTG_ECUDA;
    if (!g->exec || g->tol_newton != tol_newton || g->tol_cg != tol_cg) {
        const int rc = group_build(g, tol_newton, tol_cg);
        if (rc) return rc;
    }
    // inputs: per handle the run mask, dE and the committed E
    std::vector<int> runs(total, 1);
    if (run)
        for (size_t i = 0; i < total; ++i) runs[i] = run[i] ? 1 : 0;
    size_t off = 0;
    for (fftg_handle* h : g->hs) {
        const int B = h->B;
        if (cudaMemcpyAsync(h->run_dev, runs.data() + off, B * sizeof(int), cudaMemcpyHostToDevice, g->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(h->dE_dev, dE + 6 * off, (size_t)B * 48, cudaMemcpyHostToDevice, g->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(h->Ecom_dev, h->E.data(), (size_t)B * 48, cudaMemcpyHostToDevice, g->stream) !=
                cudaSuccess)
            return FFTG_ECUDA;
        off += (size_t)B;
    }
    if (cudaGraphLaunch(g->exec, g->stream) != cudaSuccess) return FFTG_ECUDA;
    for (size_t k = 0; k < g->hs.size(); ++k) {
        fftg_handle* h = g->hs[k];
        if (cudaMemcpyAsync(g->h_inc[k].data(), h->inc_dev, (size_t)h->B * sizeof(IncDev),
                            cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
            return FFTG_ECUDA;
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return FFTG_ECUDA;
    int first = FFTG_OK;
    off = 0;
    for (size_t k = 0; k < g->hs.size(); ++k) {
        fftg_handle* h = g->hs[k];
        int max_newton = 0, max_cg = 0;
        for (int b = 0; b < h->B; ++b, ++off) {
            const IncDev& s = g->h_inc[k][b];
            const bool on = runs[off] != 0;
            reset_stats(h, b);
            fftg_stats& st = h->stats[b];
            st.newton_iters = s.newton;
            st.cg_iters = s.cg;
            st.status = on ? (s.state == INC_DONE ? FFTG_OK : s.state == INC_FAILED ? s.status : FFTG_ENOCONV_NEWTON)
                           : FFTG_OK;
            status[off] = st.status;
            if (newton_iters) newton_iters[off] = s.newton;
            if (cg_iters) cg_iters[off] = s.cg;
            if (on && s.state == INC_DONE) {
                for (int c = 0; c < 6; ++c) {
                    sigma_out[6 * off + c] = s.sigma[c];
                    h->E[6 * b + c] += dE[6 * off + c];
                }
                h->have_tangent[b] = 1;
                h->have_update[b] = 1;
            }
            if (on && st.status != FFTG_OK && first == FFTG_OK) first = st.status;
            max_newton = std::max(max_newton, s.newton);
            max_cg = std::max(max_cg, s.cg);
        }
        // kernels of the branch: begin, end, commit, the commit's stress
        // update; per Newton pass 15 outside the CG loop; per CG loop pass
        // the iteration's kernels and the loop test (an upper bound when
        // the cells' CG counts differ between Newton passes)
        const long long per_cg = 7;
        h->launches += 4 + 15LL * max_newton + (per_cg + 1) * (max_cg + max_newton);
        g->launches += 4 + 15LL * max_newton + (per_cg + 1) * (max_cg + max_newton);
    }
    return first;
}

long long fftg_group_launch_count(const fftg_group* g) { return g ? g->launches : 0; }


void fftg_default_options(fftg_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = FFTG_MIXED;
    o->max_newton = 50;
    o->max_cg = 2000;
    o->cg_inner_floor = 1e-5;
    o->nrhs_tangent = 6;
    o->cg_graph = 1;
    o->dt = 1.0;
}

const char* fftg_version(void) { return "fftg 0.4 (sm_103a)"; }

int fftg_workspace_size_batch(int N, int ncells, const fftg_options* opt, size_t* bytes) {
    if (!bytes || !valid_grid(N) || ncells < 1) return FFTG_EINVAL;
    fftg_options o;
    if (opt) o = *opt; else fftg_default_options(&o);
    if (o.nrhs_tangent != 0 && o.nrhs_tangent != 6) return FFTG_EINVAL;
    *bytes = make_layout(N, o.precision == FFTG_MIXED, o.nrhs_tangent, ncells).total;
    return FFTG_OK;
}

int fftg_workspace_size(int N, const fftg_options* opt, size_t* bytes) {
    return fftg_workspace_size_batch(N, 1, opt, bytes);
}

int fftg_create_batch(fftg_handle** out, int N, int ncells, const uint8_t* phase, int nphase,
                      const fftg_phase* mats, const fftg_options* opt) {
    if (!out || !phase || !mats || nphase < 1 || nphase > 256 || !valid_grid(N) || ncells < 1)
        return FFTG_EINVAL;
    *out = nullptr;
    fftg_options o;
    if (opt) o = *opt; else fftg_default_options(&o);
    if ((o.precision != FFTG_FP64 && o.precision != FFTG_MIXED) || o.max_newton < 1 || o.max_cg < 1 ||
        (o.nrhs_tangent != 0 && o.nrhs_tangent != 6) || o.fixed_cg < 0 || o.fixed_newton < 0 ||
        !fftg::pos_finite(o.dt) || (o.solver != FFTG_SOLVER_CG && o.solver != FFTG_SOLVER_RICHARDSON))
        return FFTG_EINVAL;
    for (int i = 0; i < nphase; ++i)
        if (!fftg::phase_valid(mats[i], true)) return FFTG_EINVAL;
    const size_t V = (size_t)N * N * N;
    for (size_t v = 0; v < V * (size_t)ncells; ++v)
        if (phase[v] >= nphase) return FFTG_EINVAL;

    fftg_handle* h = new (std::nothrow) fftg_handle();
    if (!h) return FFTG_ENOMEM;
    h->N = N;
    h->V = (long long)V;
    h->cs = comp_stride(N);
    h->H = (N + 1) / 2;
    h->mixed = o.precision == FFTG_MIXED;
    h->nrhs = o.nrhs_tangent;
    h->B = ncells;
    h->nf = std::max(ncells, std::max(1, h->nrhs));
    h->opt = o;
    h->stream = (cudaStream_t)o.stream;
    h->nphase = nphase;
    h->E.assign((size_t)6 * ncells, 0.0);
    h->have_tangent.assign(ncells, 0);
    h->have_update.assign(ncells, 0);
    h->stats.assign(ncells, fftg_stats{});
    const Layout L = make_layout(N, h->mixed, h->nrhs, ncells);
    if (o.workspace) {
        if (o.workspace_bytes < L.total || ((uintptr_t)o.workspace & 255u)) {
            delete h;
            return FFTG_ENOMEM;
        }
        h->ws = (char*)o.workspace;
        h->own_ws = false;
    } else {
        if (cudaMalloc((void**)&h->ws, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return FFTG_ENOMEM;
        }
        h->own_ws = true;
    }
    h->ws_bytes = L.total;
    h->phase = (uint8_t*)(h->ws + L.off_phase);
    h->mats = (double*)(h->ws + L.off_mats);
    h->eps_star = (double*)(h->ws + L.off_eps_star);
    h->eps_work = (double*)(h->ws + L.off_eps_work);
    h->eps_p = (double*)(h->ws + L.off_eps_p);
    h->eps_p_tr = (double*)(h->ws + L.off_eps_p_tr);
    h->epbar = (double*)(h->ws + L.off_epbar);
    h->epbar_tr = (double*)(h->ws + L.off_epbar_tr);
    h->sigma = (double*)(h->ws + L.off_sigma);
    h->tangent = h->ws + L.off_tangent;
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
    h->nd = (NewtonDev*)(h->ws + L.off_nd);
    h->Edev = (double*)(h->ws + L.off_E);
    h->active = (int*)(h->ws + L.off_active);
    h->out36 = (double*)(h->ws + L.off_out36);
    h->guard = (unsigned int*)(h->ws + L.off_guard);
    h->run_dev = (int*)(h->ws + L.off_run);
    h->dE_dev = (double*)(h->ws + L.off_dE);
    h->Ecom_dev = (double*)(h->ws + L.off_Ecom);
    h->fin_dev = (int*)(h->ws + L.off_fin);
    h->inc_dev = (IncDev*)(h->ws + L.off_inc);

    auto fail = [&](int code) {
        fftg_destroy(h);
        return code;
    };
    if (cudaMallocHost((void**)&h->h_cg, h->nf * sizeof(CGState)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_nd, ncells * sizeof(NewtonDev)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_out36, 36 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_E, (size_t)ncells * 6 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&h->h_active, ncells * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FFTG_ENOMEM);
    }
    std::vector<double> tw64(2 * N);
    std::vector<float> tw32(2 * N), twdd(4 * N);
    twiddles(N, tw64.data(), tw32.data(), twdd.data());
    std::vector<double> m(fftg::kMatStride * nphase);
    for (int i = 0; i < nphase; ++i) fftg::pack_phase(mats[i], &m[fftg::kMatStride * i]);
    cudaStream_t s = h->stream;
    bool ok = true;
    for (int b = 0; b < ncells && ok; ++b)
        ok = cudaMemcpyAsync(h->phase + (size_t)b * h->cs, phase + (size_t)b * V, V, cudaMemcpyHostToDevice,
                             s) == cudaSuccess;
    if (!ok || cudaMemcpyAsync(h->mats, m.data(), m.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->tw64, tw64.data(), tw64.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->tw32, tw32.data(), tw32.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->twdd, twdd.data(), twdd.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(h->eps_star, 0, (size_t)ncells * 6 * h->cs * 8, s) != cudaSuccess ||
        cudaMemsetAsync(h->eps_p, 0, (size_t)ncells * 6 * h->cs * 8, s) != cudaSuccess ||
        cudaMemsetAsync(h->epbar, 0, (size_t)ncells * h->cs * 8, s) != cudaSuccess ||
        cudaMemsetAsync(h->cg, 0, h->nf * sizeof(CGState), s) != cudaSuccess ||
        cudaMemsetAsync(h->nd, 0, ncells * sizeof(NewtonDev), s) != cudaSuccess ||
        cudaMemsetAsync(h->Edev, 0, (size_t)ncells * 6 * 8, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        h->last_cuda = cudaGetLastError();
        return fail(FFTG_ECUDA);
    }
    *out = h;
    return FFTG_OK;
}

int fftg_create(fftg_handle** out, int N, const uint8_t* phase, int nphase, const fftg_phase* mats,
                const fftg_options* opt) {
    return fftg_create_batch(out, N, 1, phase, nphase, mats, opt);
}

void fftg_destroy(fftg_handle* h) {
    if (!h) return;
    if (h->stream || h->ws) cudaStreamSynchronize(h->stream);
    free_graphs(h);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->h_cg) cudaFreeHost(h->h_cg);
    if (h->h_nd) cudaFreeHost(h->h_nd);
    if (h->h_out36) cudaFreeHost(h->h_out36);
    if (h->h_E) cudaFreeHost(h->h_E);
    if (h->h_active) cudaFreeHost(h->h_active);
    if (h->prof) {
        for (int i = 0; i < Prof::kRing; ++i) {
            if (h->prof->ev0[i]) cudaEventDestroy(h->prof->ev0[i]);
            if (h->prof->ev1[i]) cudaEventDestroy(h->prof->ev1[i]);
        }
        delete h->prof;
    }
    delete h;
}

int fftg_batch_size(const fftg_handle* h) { return h ? h->B : 0; }

int fftg_select_cell(fftg_handle* h, int cell) {
    if (!h || cell < 0 || cell >= h->B) return FFTG_EINVAL;
    h->sel = cell;
    return FFTG_OK;
}

int fftg_profile_kinds(void) { return KK_COUNT; }

const char* fftg_profile_name(int kind) {
    return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : nullptr;
}

int fftg_profile_enable(fftg_handle* h, int on) {
    if (!h) return FFTG_EINVAL;
    if (on && !h->prof) {
        h->prof = new (std::nothrow) Prof();
        if (!h->prof) return FFTG_ENOMEM;
        for (int i = 0; i < Prof::kRing; ++i) {
            CK(cudaEventCreate(&h->prof->ev0[i]));
            CK(cudaEventCreate(&h->prof->ev1[i]));
        }
    }
    if (h->prof) {
        CK(prof_drain(h));
        h->prof->on = on != 0;
    }
    return FFTG_OK;
}

int fftg_profile_reset(fftg_handle* h) {
    if (!h) return FFTG_EINVAL;
    if (h->prof) {
        CK(prof_drain(h));
        for (int k = 0; k < KK_COUNT; ++k) {
            h->prof->ms[k] = 0.0;
            h->prof->cnt[k] = 0;
        }
    }
    return FFTG_OK;
}

int fftg_profile_read(fftg_handle* h, int kind, double* total_ms, long long* launches) {
    if (!h || kind < 0 || kind >= KK_COUNT) return FFTG_EINVAL;
    if (h->prof) CK(prof_drain(h));
    if (total_ms) *total_ms = h->prof ? h->prof->ms[kind] : 0.0;
    if (launches) *launches = h->prof ? h->prof->cnt[kind] : 0;
    return FFTG_OK;
}

long long fftg_launch_count(const fftg_handle* h) { return h ? h->launches : 0; }

int fftg_batch_step(fftg_handle* h, const double* dE, double tol_newton, double tol_cg, double* sigma_out,
                    int* newton_iters, int* cg_iters, int* status) {
    if (!h || !dE || !sigma_out || !status || !(tol_newton > 0) || !(tol_cg > 0)) return FFTG_EINVAL;
    for (int k = 0; k < 6 * h->B; ++k)
        if (!std::isfinite(dE[k])) return FFTG_ENAN;
    return batch_step(h, dE, tol_newton, tol_cg, sigma_out, newton_iters, cg_iters, status);
}

int fftg_step(fftg_handle* h, const double dE[6], double tol_newton, double tol_cg, double sigma_out[6],
              int* newton_iters, int* cg_iters) {
    if (!h || !dE || !sigma_out || !(tol_newton > 0) || !(tol_cg > 0)) return FFTG_EINVAL;
    if (h->B != 1) return FFTG_EINVAL;
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(dE[c])) return FFTG_ENAN;
    int st = 0;
    return batch_step(h, dE, tol_newton, tol_cg, sigma_out, newton_iters, cg_iters, &st);
}

int fftg_last_stats(fftg_handle* h, fftg_stats* out) {
    if (!h || !out) return FFTG_EINVAL;
    *out = h->stats[h->sel];
    return FFTG_OK;
}

int fftg_tangent(fftg_handle* h, double tol_cg, double C_out[36], int* cg_iters) {
    if (!h || !C_out || !(tol_cg > 0)) return FFTG_EINVAL;
    if (h->nrhs != 6) return FFTG_EINVAL;
    const int cell = h->sel;
    if (!h->have_tangent[cell]) return FFTG_ESTATE;
    const bool f64 = !h->mixed;
    const size_t ts = f64 ? 8 : 4;
    const void* tg = (const char*)h->tangent + (size_t)cell * 7 * h->cs * ts;
    const double tol = h->mixed ? std::max(tol_cg, h->opt.cg_inner_floor) : tol_cg;
    set_cg_params(h, 6, tol, nullptr);
    CK(cudaMemcpyAsync(h->cg, h->h_cg, h->nf * sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
    VecArgs u{};
    u.V = h->V;
    u.cs = h->cs;
    u.tangent = tg;
    u.cg = h->cg;
    u.nd = h->nd;
    u.partials = h->partials;
    u.fstride = 6 * h->cs;
    const int nb = pointwise_blocks(h->V);
    int slot = prof_begin(h, KK_TANGENT_FLOOR);
    if (f64)
        k_tangent_floor<double><<<nb, kThreads, 0, h->stream>>>(u);
    else
        k_tangent_floor<float><<<nb, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    PassArgs a = base_args(h, f64);
    a.tangent = tg;
    a.out = h->spec;
    CK(pass(h, f64 ? PK_P1_TANRHS_F64 : PK_P1_TANRHS_F32, a, 6));
    int rc = run_p234(h, f64 ? FFT_F64 : FFT_F32, -invN3, nullptr, 6, nullptr);
    if (rc) return rc;
    PassArgs b = base_args(h, f64);
    b.in = h->spec;
    b.out = h->r;
    b.cg = h->cg;
    CK(pass(h, f64 ? PK_P5_RHS_F64_TO_F64 : PK_P5_RHS_F32_TO_F32, b, 6));
    CK(cudaMemsetAsync(h->x, 0, 6 * 6 * h->cs * ts, h->stream));
    rc = launch_bounds(h, tg, 0, 1, 6, nullptr);
    if (rc) return rc;
    rc = run_cg(h, 6, tg, 0);
    if (rc) return rc;
    rc = project_solution(h, 6, nullptr);
    if (rc) return rc;
    int total = 0;
    for (int f = 0; f < 6; ++f) {
        if (h->h_cg[f].done == CG_BREAKDOWN) return FFTG_ENAN;
        total += h->h_cg[f].it;
    }
    u.x = h->x;
    u.out = h->out36;
    slot = prof_begin(h, KK_TANGENT_AVERAGE);
    if (f64)
        k_tangent_average<double><<<nb, kThreads, 0, h->stream>>>(u);
    else
        k_tangent_average<float><<<nb, kThreads, 0, h->stream>>>(u);
    prof_end(h, slot);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_out36, h->out36, 36 * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 36; ++k) C_out[k] = h->h_out36[k] / (double)h->V;
    if (cg_iters) *cg_iters = total;
    return FFTG_OK;
}

size_t fftg_state_bytes(const fftg_handle* h) {
    if (!h) return 0;
    return (size_t)(6 + 13 * h->V) * sizeof(double);
}

int fftg_get_state(fftg_handle* h, void* buf, size_t bytes) {
    if (!h || !buf || bytes < fftg_state_bytes(h)) return FFTG_EINVAL;
    return download_cell(h, h->sel, (double*)buf);
}

int fftg_set_state(fftg_handle* h, const void* buf, size_t bytes) {
    if (!h || !buf || bytes < fftg_state_bytes(h)) return FFTG_EINVAL;
    const double* d = (const double*)buf;
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(d[c])) return FFTG_EINVAL;
    return upload_cell(h, h->sel, nullptr, d);
}

int fftg_reset_state(fftg_handle* h) {
    if (!h) return FFTG_EINVAL;
    return upload_cell(h, h->sel, nullptr, nullptr);
}

int fftg_get_field(fftg_handle* h, int which, double* out) {
    if (!h || !out) return FFTG_EINVAL;
    const size_t V = (size_t)h->V;
    const int cell = h->sel;
    switch (which) {
        case FFTG_FIELD_STRAIN: {
            CK(copy_field(h, out, false, cell_field(h->eps_star, h, cell), true, 8, cudaMemcpyDeviceToHost));
            CK(cudaStreamSynchronize(h->stream));
            for (int c = 0; c < 6; ++c)
                for (size_t v = 0; v < V; ++v) out[c * V + v] += h->E[6 * cell + c];
            return FFTG_OK;
        }
        case FFTG_FIELD_STRESS: {
            // The committed plastic strain is the return-mapped one at the
            // committed strain, so the converged stress is C_e : (eps -
            // eps_p) there: the stress update runs with the return skipped
            // (a visco-plastic phase has no elastic range, and a second
            // return would relax the stress again). Non-linear elastic
            // phases have no history and are evaluated as usual. The tangent
            // of the increment is left untouched.
            std::memcpy(h->h_E + 6 * cell, h->E.data() + 6 * cell, 6 * sizeof(double));
            CK(cudaMemcpyAsync(h->Edev + 6 * cell, h->h_E + 6 * cell, 48, cudaMemcpyHostToDevice, h->stream));
            int rc = launch_constitutive(h, nullptr, 1, cell, h->eps_star, h->sigma, false, nullptr, false, true);
            if (rc) return rc;
            CK(copy_field(h, out, false, cell_field(h->sigma, h, cell), true, 8, cudaMemcpyDeviceToHost));
            CK(cudaStreamSynchronize(h->stream));
            return FFTG_OK;
        }
        case FFTG_FIELD_EPBAR:
            CK(cudaMemcpyAsync(out, h->epbar + (size_t)cell * h->cs, V * 8, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            return FFTG_OK;
        case FFTG_FIELD_EPS_P:
            CK(copy_field(h, out, false, cell_field(h->eps_p, h, cell), true, 8, cudaMemcpyDeviceToHost));
            CK(cudaStreamSynchronize(h->stream));
            return FFTG_OK;
        case FFTG_FIELD_TANGENT: {
            if (!h->have_update[cell]) return FFTG_ESTATE;
            const size_t ts = h->mixed ? 4 : 8;
            const char* tg = (const char*)h->tangent + (size_t)cell * 7 * h->cs * ts;
            if (!h->mixed) {
                CK(copy_field(h, out, false, tg, true, 8, cudaMemcpyDeviceToHost, 7));
                CK(cudaStreamSynchronize(h->stream));
                return FFTG_OK;
            }
            std::vector<float> tmp(7 * V);
            CK(copy_field(h, tmp.data(), false, tg, true, 4, cudaMemcpyDeviceToHost, 7));
            CK(cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < 7 * V; ++i) out[i] = (double)tmp[i];
            return FFTG_OK;
        }
        default:
            return FFTG_EINVAL;
    }
}

int fftg_op_project(fftg_handle* h, int precision, const void* tau, void* out) {
    if (!h || !tau || !out || (precision != FFTG_FP64 && precision != FFTG_MIXED && precision != FFTG_DD))
        return FFTG_EINVAL;
    const int prec = precision == FFTG_FP64 ? FFT_F64 : precision == FFTG_DD ? FFT_DD : FFT_F32;
    const bool f64 = prec != FFT_F32;  // FP64 buffers (FFTG_FP64, FFTG_DD)
    const size_t es = f64 ? 8 : 4;
    // internal scratch in the padded layout: FP64 in sigma / eps_work, FP32
    // in p / q (these hold no state between increments)
    void* in_buf = f64 ? (void*)h->sigma : h->p;
    void* out_buf = f64 ? (void*)h->eps_work : h->q;
    CK(copy_field(h, in_buf, true, tau, false, es, cudaMemcpyDeviceToDevice));
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    PassArgs a = base_args_fft(h, prec);
    a.in = in_buf;
    a.out = h->spec;
    CK(pass(h, prec == FFT_DD ? PK_P1_PLAIN_DD : f64 ? PK_P1_PLAIN_F64 : PK_P1_PLAIN_F32, a, 1));
    int rc = run_p234(h, prec, invN3, nullptr, 1, nullptr);
    if (rc) return rc;
    PassArgs b = base_args_fft(h, prec);
    b.in = h->spec;
    b.out = out_buf;
    CK(pass(h, prec == FFT_DD ? PK_P5_PLAIN_DD_TO_F64 : f64 ? PK_P5_PLAIN_F64 : PK_P5_PLAIN_F32, b, 1));
    CK(copy_field(h, out, false, out_buf, true, es, cudaMemcpyDeviceToDevice));
    return FFTG_OK;
}

int fftg_op_constitutive(fftg_handle* h, const double dE[6], const double* eps, double* sigma) {
    if (!h) return FFTG_EINVAL;
    const int cell = h->sel;
    for (int c = 0; c < 6; ++c) h->h_E[6 * cell + c] = h->E[6 * cell + c] + (dE ? dE[c] : 0.0);
    CK(cudaMemcpyAsync(h->Edev + 6 * cell, h->h_E + 6 * cell, 48, cudaMemcpyHostToDevice, h->stream));
    const double* e = h->eps_star;
    if (eps) {
        CK(copy_field(h, cell_field(h->eps_work, h, cell), true, eps, false, 8, cudaMemcpyDeviceToDevice));
        e = h->eps_work;
    }
    int rc = launch_constitutive(h, nullptr, 1, cell, e, h->sigma, false, nullptr);
    if (rc) return rc;
    if (sigma)
        CK(copy_field(h, sigma, false, cell_field(h->sigma, h, cell), true, 8, cudaMemcpyDeviceToDevice));
    h->have_tangent[cell] = 0;
    return FFTG_OK;
}

int fftg_op_matvec(fftg_handle* h, int precision, const void* p, void* q, double* pq) {
    if (!h || !p || !q) return FFTG_EINVAL;
    const bool f64 = precision == FFTG_FP64;
    if (f64 == (bool)h->mixed) return FFTG_EINVAL;  // must match the tangent's precision
    const size_t es = f64 ? 8 : 4;
    set_cg_params(h, 1, 1.0, nullptr);
    h->h_cg[0].rr = 1.0;
    CK(cudaMemcpyAsync(h->cg, h->h_cg, h->nf * sizeof(CGState), cudaMemcpyHostToDevice, h->stream));
    CK(copy_field(h, h->p, true, p, false, es, cudaMemcpyDeviceToDevice));
    const double invN3 = 1.0 / ((double)h->N * h->N * h->N);
    PassArgs a = base_args(h, f64);
    a.in = h->p;
    a.tangent = (const char*)h->tangent + (size_t)h->sel * 7 * h->cs * es;
    a.out = h->spec;
    CK(pass(h, f64 ? PK_P1_TAN_F64 : PK_P1_TAN_F32, a, 1));
    int rc = run_p234(h, f64 ? FFT_F64 : FFT_F32, invN3, nullptr, 1, nullptr);
    if (rc) return rc;
    PassArgs b = base_args(h, f64);
    b.in = h->spec;
    b.out = h->q;
    b.aux = h->p;
    b.cg = h->cg;
    CK(pass(h, f64 ? PK_P5_DOT_F64 : PK_P5_DOT_F32, b, 1));
    CK(copy_field(h, q, false, h->q, true, es, cudaMemcpyDeviceToDevice));
    if (pq) {
        CK(cudaMemcpyAsync(h->h_cg, h->cg, sizeof(CGState), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *pq = h->h_cg[0].pq;
    }
    return FFTG_OK;
}

}  // extern "C"
