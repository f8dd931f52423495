// The five grid passes of the projected matvec q = G (C : p) and of the
// residual G sigma, on a real field [nf][6][N][N][N] and a half spectrum
// [nf][6][N][N][H], H = (N+1)/2 (odd N: no Nyquist mode, Section 2.3).
//
//   P1 (rows, x3)  [p = r + beta p]; tau = C : p (Section 4.2 tangent) or
//                  tau = input; real-to-complex FFT along x3: two real
//                  components share one complex FFT and are split after it
//   P2 (x2)        complex FFT along x2
//   P3 (x1)        complex FFT along x1, Ghat (Appendix A, Eq. FT_projection,
//                  in the closed form n(x)(tau n) + (tau n)(x)n - (n.tau n) n(x)n)
//                  times the forward 1/|N| factor, inverse FFT along x1
//   P4 (x2)        inverse complex FFT along x2
//   P5 (rows, x3)  complex-to-real inverse FFT along x3; writes q and the
//                  block partials of <p, q> (or the CG right-hand side)
//
// Together: G tau = F^-1 [Ghat : F[tau]], Eq. (discrete_projection).
#pragma once

#include "common.cuh"
#include "dd.cuh"
#include "fft_core.cuh"

namespace fftg {

enum : int { P1_PLAIN = 0, P1_TAN = 1, P1_CG = 2, P1_TANRHS = 3, P1_CGF = 4 };
enum : int { P5_PLAIN = 0, P5_DOT = 1, P5_RHS = 2, P5_CGF = 3 };

// The two CG iterations of the passes.
//
// P1_CG / P5_DOT (+ the update kernel): Hestenes-Stiefel CG on G C as
// written, alpha = <r, r> / <p, G C p> from the product of P5, then
// r -= alpha q and <r, r> in a separate pass over r and q.
//
// P1_CGF / P5_CGF (mixed path): on compatible fields G is the orthogonal
// projector onto them, so <p, G C p> = <G p, C p> = <p, C p>; P1 forms
// C : p anyway and reduces <p, C : p> there, so alpha is known before P5,
// which then updates r -= alpha q with q still in registers and reduces
// <r, r>: q is never stored and the update pass disappears (72 B per voxel
// and field less per iteration in FP32). The iterates are those of CG up to
// the rounding of the incompatible part that the FP32 recursion leaves in p
// (about 1e-5 of |p| after some tens of iterations, removed by the
// projection of each inner solution).

struct PassArgs {
    const void* in;        // P1: real field; P2-P4: unused; P5: spectrum
    void* out;             // P1: spectrum; P2-P4: spectrum (in place); P5: real field
    const void* aux;       // P1_CG: r; P5_DOT: p
    void* aux2;            // P1_CG: p (updated in place)
    void* aux3;            // P1_CG: x (gets the previous iteration's alpha p);
                           // P5_CGF: r (updated in place; aux is the same r)
    const void* tangent;   // [7][V]: K', 2G_eff, w11, w22, w23, w13, w12 (see apply_tangent7)
    CGState* cg;           // per field, or null
    double* partials;      // [nf][nblocks][2]
    const void* tw;        // w_N^j, j < N, in the FFT precision
    double scale;          // P3: factor on Ghat (+-1/N^3)
    long long cs;          // component stride of real fields and of the tangent
                           // (elements; >= N^3 + 4, a multiple of 32)
    long long fstride;     // real-field stride between fields (elements)
    long long sstride;     // spectrum stride between fields (complex elements)
    long long tstride;     // tangent stride between fields (0: shared)
    const int* active;     // per field: 0 = skip this field (null: all run)
    // P2 of the fused CG iteration: the block partials of <p, C : p> that P1
    // wrote ([nf][red_n]); block (0, 0) of each field reduces them in a
    // fixed order and sets alpha (null: nothing to reduce)
    const double* red_in;
    int red_n;
};

// Tuning of the elementwise phases of P1 and P5: voxels per lane (1, 2 or 4,
// moved as one vector per component) and the minimum resident blocks per SM
// (an upper bound on registers). Chosen by timing the variants at 243^3:
// P1 with 4 voxels per lane and 3 blocks per SM (80 registers) took 0.355 ms
// per CG iteration against 0.44 ms (1 block) and 0.39 ms (2 voxels, 4 blocks):
// its 19 loads per voxel need many bytes in flight. P5 with 2 voxels per
// lane and 4 blocks per SM took 0.223 ms against 0.245 (1 or 4 voxels) and
// 0.31-0.38 ms with 2 blocks per SM.
#ifndef FFTG_P1_VW
#define FFTG_P1_VW 4
#endif
#ifndef FFTG_P1_MINB
#define FFTG_P1_MINB 3
#endif
#ifndef FFTG_P5_VW
#define FFTG_P5_VW 2
#endif
#ifndef FFTG_P5_MINB
#define FFTG_P5_MINB 4
#endif
// P5: rounds of spectrum loads (LDB) and of p loads (PB) issued together,
// so that more loads are in flight per thread: at 243^3 LDB = 4, PB = 2
// took P5 from 0.177 to 0.157 ms (PB = 4 or one voxel per lane: no further
// gain; 3 blocks per SM instead of 4: 0.173 ms).
#ifndef FFTG_P5_LDB
#define FFTG_P5_LDB 4
#endif
#ifndef FFTG_P5_PB
#define FFTG_P5_PB 2
#endif

#ifndef FFTG_P3_TB
#define FFTG_P3_TB 1
#endif

// Double-float passes (the mixed path's residual): P3 columns per block
// (0 = the rule in Cfg) and minimum resident blocks per SM of P1/P5 and of
// P3. At 243^3 one block per SM for P1/P5 (more registers) took them from
// 2.05/1.56 to 3.42/2.66 ms; three spill.
#ifndef FFTG_DD_P3_W
#define FFTG_DD_P3_W 0
#endif
#ifndef FFTG_DD_MINB
#define FFTG_DD_MINB 2
#endif
#ifndef FFTG_DD_P3_MINB
#define FFTG_DD_P3_MINB 1
#endif

template <typename T>
constexpr bool is_dd_v = std::is_same<T, dd>::value;

// Block shapes: P3 columns per block (0 = as many as fit ~100 KB of shared
// memory, at most 32) and P1/P5 rows per block (0 = as many as fit ~50 KB,
// at least 4).
#ifndef FFTG_P3_W
#define FFTG_P3_W 0
#endif
#ifndef FFTG_ROWS
#define FFTG_ROWS 0
#endif

template <typename T, int W>
struct VecN;
template <typename T>
struct VecN<T, 1> {
    using type = T;
};
template <>
struct VecN<float, 2> {
    using type = float2;
};
template <>
struct VecN<float, 4> {
    using type = float4;
};
template <>
struct VecN<double, 2> {
    using type = double2;
};
template <>
struct VecN<dd, 2> {
    using type = float4;
};

template <int W, typename T>
__device__ __forceinline__ void ldv(const T* p, T (&v)[W]) {
    using VT = typename VecN<T, W>::type;
    const VT t = *reinterpret_cast<const VT*>(p);
    const T* e = reinterpret_cast<const T*>(&t);
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = e[k];
}
template <int W, typename T>
__device__ __forceinline__ void stv(T* p, const T (&v)[W]) {
    using VT = typename VecN<T, W>::type;
    VT t;
    T* e = reinterpret_cast<T*>(&t);
#pragma unroll
    for (int k = 0; k < W; ++k) e[k] = v[k];
    *reinterpret_cast<VT*>(p) = t;
}

// Block shapes of the passes for the radix split N = NA * (N / NA) and the
// tile variant TV (the autotuner's schedules; NA = Plan<N>::N1, TV = 0 are
// the defaults): P1/P5 rows per block R (TV 1: half, 2: double), P3
// columns per block W3 (TV 1: half, 2: double, within the shared memory of
// a block), P2/P4 columns per block W2 (FP32, TV 1: 32 instead of 16).
template <int N, typename T, int NA = Plan<N>::N1, int TV = 0>
struct Cfg {
    static constexpr int PN1 = NA, PN2 = N / NA;
    static constexpr int H = (N + 1) / 2;
    static constexpr int CS = (int)sizeof(cplx<T>);
    static constexpr int BUDGET = 100 * 1024;
    static constexpr int ROW_BUDGET = 50 * 1024;
    static constexpr int SMEM_MAX = 227 * 1024;
    static constexpr int fl2(int x) {
        return x >= 64 ? 64 : x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1;
    }
    // rows per block in P1/P5: a power of two >= 4, so that a block's rows
    // are a whole number of 16-byte vectors
    static constexpr int R0 = FFTG_ROWS > 0 ? FFTG_ROWS : fl2(ROW_BUDGET / (3 * N * CS));
    static constexpr int R1 = R0 < 4 ? 4 : R0;
    static constexpr int R = TV == 1 ? (R1 / 2 < 4 ? 4 : R1 / 2)
                             : TV == 2 && (size_t)(3 * 2 * R1 * N + N) * CS <= SMEM_MAX ? 2 * R1 : R1;
    // voxels per lane in P1's elementwise phase (FP64: at most 2 = 16 bytes)
    static constexpr int VW = (sizeof(T) == 8 && FFTG_P1_VW > 2) ? 2 : FFTG_P1_VW;
    static constexpr int W3a = fl2(BUDGET / (6 * N * CS)) > 32 ? 32 : fl2(BUDGET / (6 * N * CS));
    // double-float P3: up to twice the shared memory, as long as the block
    // keeps <= 512 threads (so <= 128 registers each): at 243^3 8 columns
    // took the pass from 3.35 to 2.29 ms against 4 (the FP64 rule); 2
    // columns 3.33 ms
    static constexpr int WDa = fl2(2 * BUDGET / (6 * N * CS)) > 32 ? 32 : fl2(2 * BUDGET / (6 * N * CS));
    static constexpr int WDt = PN2 == 1 ? 32
                               : (fl2(512 / (6 * PN2)) < fl2(512 / (2 * PN1))
                                      ? fl2(512 / (6 * PN2))
                                      : fl2(512 / (2 * PN1)));
    static constexpr int WD = WDa < WDt ? WDa : WDt;
    static constexpr int W3d = is_dd_v<T> ? (FFTG_DD_P3_W > 0 ? FFTG_DD_P3_W : (WD > W3a ? WD : W3a))
                               : (FFTG_P3_W > 0 && FFTG_P3_W < W3a) ? FFTG_P3_W : W3a;
    static constexpr int rup32(int x) { return ((x + 31) / 32) * 32; }
    static constexpr int cap(int x) { return x > 1024 ? 1024 : x; }
    static constexpr bool p3_fits(int w) {
        return (size_t)(6 * w * N + N) * CS <= SMEM_MAX && rup32(6 * w * PN2) <= 1024 &&
               rup32(2 * w * PN1) <= 1024;
    }
    static constexpr int W3 = TV == 1 ? (W3d / 2 < 1 ? 1 : W3d / 2)
                              : TV == 2 && W3d < 32 && p3_fits(2 * W3d) ? 2 * W3d : W3d;
    static constexpr int W2 = (CS == 8) ? (TV == 1 ? 32 : 16) : 32;         // columns, P2/P4
    static constexpr int S2 = fl2(BUDGET / (N * W2 * CS)) > 16 ? 16 : fl2(BUDGET / (N * W2 * CS));
    // threads of the column passes: one stage-A item per thread
    static constexpr int T2 = cap(rup32(S2 * W2 * PN2));
    // P3: one stage-A item per thread, and (FFTG_P3_TB) at least 2*W*N1
    // threads (448 at 243^3 rather than 432: the configuration measured)
    static constexpr int T3a = rup32(6 * W3 * PN2);
    static constexpr int T3b = FFTG_P3_TB ? rup32(2 * W3 * PN1) : 0;
    // single-stage plans (N2 = 1) loop over the middle stages with 256 threads
    static constexpr int T3 = PN2 == 1 ? (T3a > 256 ? cap(T3a) : 256) : cap(T3a > T3b ? T3a : T3b);
    static constexpr size_t smem_rows = (size_t)(3 * R * N + N) * CS;
    static constexpr size_t smem_p3 = (size_t)(6 * W3 * N + N) * CS;
    static constexpr size_t smem_p24 = (size_t)(S2 * W2 * N + N) * CS;
    static constexpr int row_blocks = (N * N + R - 1) / R;
};

// Real type a plain P1 reads: the FFT type, except for double-float FFTs,
// whose input is an FP64 field (split into hi + lo on load).
template <typename T>
struct PlainIn {
    using type = T;
};
template <>
struct PlainIn<dd> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ void load_tw(cplx<T>* tw, const void* src, int n) {
    const cplx<T>* s = (const cplx<T>*)src;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = s[i];
}

// s = C : p with the compact J2 tangent (Section 4.2):
// C = |K'| I(x)I + 2G_eff I_d + b N(x)N, stored as w = sqrt(|b|) N and the
// sign of b in the sign of K' (K > 0): K' > 0 for b <= 0, always the case
// for hardening exponents n <= 1; K' < 0 for b > 0. w33 = -(w11 + w22).
template <typename T>
__device__ __forceinline__ void apply_tangent7(T K, T g2, T w0, T w1, T w3, T w4, T w5,
                                               const T (&p)[6], T (&s)[6]) {
    const T w2 = -(w0 + w1);
    const T tr = p[0] + p[1] + p[2];
    const T m = tr * T(1.0 / 3.0);
    T wp = w0 * p[0] + w1 * p[1] + w2 * p[2] + T(2) * (w3 * p[3] + w4 * p[4] + w5 * p[5]);
    if (K < T(0)) {
        K = -K;
        wp = -wp;
    }
    const T kt = K * tr;
    s[0] = kt + g2 * (p[0] - m) - wp * w0;
    s[1] = kt + g2 * (p[1] - m) - wp * w1;
    s[2] = kt + g2 * (p[2] - m) - wp * w2;
    s[3] = g2 * p[3] - wp * w3;
    s[4] = g2 * p[4] - wp * w4;
    s[5] = g2 * p[5] - wp * w5;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
};
template <>
struct Vec16<double> {
    using type = double2;
};

// ----------------------------------------------------------------------- P1
template <int N, typename T, int MODE, int NA = Plan<N>::N1, int TV = 0>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? FFTG_P1_MINB : is_dd_v<T> ? FFTG_DD_MINB : 2)
    k_p1(PassArgs a) {
    using C = Cfg<N, T, NA, TV>;
    constexpr int R = C::R, H = C::H;
    constexpr int N1 = NA, N2 = N / NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [3][R][N]
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    constexpr bool CGM = MODE == P1_CG || MODE == P1_CGF;
    if (CGM && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const long long cs = a.cs;
    using TIn = typename PlainIn<T>::type;
    const TIn* in = (const TIn*)a.in + f * a.fstride;
    const T* tg = (const T*)a.tangent + f * a.tstride;
    T beta = T(0), alpha = T(0);
    T pcp = T(0);       // P1_CGF: this thread's part of <p, C : p>
    bool first = true;  // first CG iteration: p = r (p holds no data yet)
    if (CGM) {
        beta = (T)a.cg[f].beta;
        alpha = (T)a.cg[f].alpha;
        first = a.cg[f].it == 0;
    }
    // Elementwise phase: each lane takes VW consecutive voxels of the block's
    // R rows (R*N contiguous elements per component, R a multiple of 4, so
    // a block starts on a vector boundary) and loads them as one vector per
    // component; more voxels per lane keep more loads in flight. In the last
    // block the vector that straddles the end of the grid reads and writes
    // only the padding of the component (cs >= N^3 + 4), and its lanes past
    // the grid belong to rows that the FFT stages skip.
    constexpr int VW = C::VW;
    for (int j = tid; j < (R * N) / VW; j += kThreads) {
        const int i0 = j * VW;
        T s[6][VW];
        if (i0 < nel) {
            const long long v0 = base + i0;
            T p[6][VW];
            if (CGM) {
                // x += alpha p (the step of the previous iteration, which the
                // update left to this pass), then p = r + beta p
                const T* r = (const T*)a.aux + f * a.fstride;
                T* pp = (T*)a.aux2 + f * a.fstride;
                T* xx = (T*)a.aux3 + f * a.fstride;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    ldv<VW, T>(r + c * cs + v0, p[c]);
                    if (!first) {
                        T po[VW], xo[VW];
                        ldv<VW, T>(pp + c * cs + v0, po);
                        ldv<VW, T>(xx + c * cs + v0, xo);
#pragma unroll
                        for (int e = 0; e < VW; ++e) {
                            xo[e] += alpha * po[e];
                            p[c][e] += beta * po[e];
                        }
                        stv<VW, T>(xx + c * cs + v0, xo);
                    }
                    stv<VW, T>(pp + c * cs + v0, p[c]);
                }
            } else if (MODE == P1_TANRHS) {
#pragma unroll
                for (int c = 0; c < 6; ++c)
#pragma unroll
                    for (int e = 0; e < VW; ++e) p[c][e] = (c == f) ? T(1) : T(0);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    TIn t[VW];
                    ldv<VW, TIn>(in + c * cs + v0, t);
#pragma unroll
                    for (int e = 0; e < VW; ++e) p[c][e] = T(t[e]);
                }
            }
            if (MODE == P1_PLAIN) {
#pragma unroll
                for (int c = 0; c < 6; ++c)
#pragma unroll
                    for (int e = 0; e < VW; ++e) s[c][e] = p[c][e];
            } else {
                T t7[7][VW];
#pragma unroll
                for (int k = 0; k < 7; ++k) ldv<VW, T>(tg + k * cs + v0, t7[k]);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    const T pe[6] = {p[0][e], p[1][e], p[2][e], p[3][e], p[4][e], p[5][e]};
                    T se[6];
                    apply_tangent7<T>(t7[0][e], t7[1][e], t7[2][e], t7[3][e], t7[4][e], t7[5][e],
                                      t7[6][e], pe, se);
#pragma unroll
                    for (int c = 0; c < 6; ++c) s[c][e] = se[c];
                    if (MODE == P1_CGF && i0 + e < nel) pcp += frob<T>(pe, se);
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int e = 0; e < VW; ++e) s[c][e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            z[i0 + e] = mk(s[0][e], s[1][e]);
            z[R * N + i0 + e] = mk(s[2][e], s[3][e]);
            z[2 * R * N + i0 + e] = mk(s[4][e], s[5][e]);
        }
    }
    // P1_CGF: this block's part of <p, C : p>, lanes by shuffles, warps in
    // index order after the barrier below; P2 reduces the blocks' parts (no
    // fence or ticket at the end of every block here)
    __shared__ double pcp_warp[kThreads / 32];
    if (MODE == P1_CGF) {
        const double wv = warp_sum((double)pcp);
        if ((tid & 31) == 0) pcp_warp[tid >> 5] = wv;
    }
    __syncthreads();
    if (MODE == P1_CGF && tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += pcp_warp[w];
        a.partials[(size_t)f * gridDim.x + blockIdx.x] = t;
    }
    constexpr int NP = 3 * R;
    for (int it = tid; it < NP * N2; it += kThreads) {
        const int pc = it % NP, t = it / NP;
        if (pc % R < nrows) fwdA<N, N1, T>(z + pc * N, 1, z + pc * N, 1, t, tw);
    }
    __syncthreads();
    if (N2 > 1) {
        for (int it = tid; it < NP * N1; it += kThreads) {
            const int pc = it % NP, k1 = it / NP;
            if (pc % R < nrows) fwdB<N, N1, false, T>(z + pc * N, 1, z + pc * N, 1, k1, tw);
        }
        __syncthreads();
    }
    cplx<T>* out = (cplx<T>*)a.out + f * a.sstride;
    const long long HS = (long long)N * N * H;
    for (int it = tid; it < nrows * H; it += kThreads) {
        const int row = it / H, k = it - row * H;
        const int pk = perm_pos<N, N1>(k), pn = perm_pos<N, N1>(k == 0 ? 0 : N - k);
        const long long o = (long long)(row0 + row) * H + k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<T> zk = z[(c * R + row) * N + pk];
            const cplx<T> zn = conj(z[(c * R + row) * N + pn]);
            const cplx<T> A = half_of(zk + zn);
            const cplx<T> d = zk - zn;  // (zk - zn) / (2i) = (d.y, -d.x) / 2
            const cplx<T> B = half_of(mk(d.y, -d.x));
            out[(2 * c) * HS + o] = A;
            out[(2 * c + 1) * HS + o] = B;
        }
    }
}

// -------------------------------------------------------------- P2 / P4 (x2)
// Blocks of T2 = (slabs x columns x N2) threads: stage A is one item per
// thread; stage B takes N1/N2 rounds. A slab is one (component, x1) plane
// of the spectrum; NC components (6 here, 9 in the finite-strain passes).
template <int N, typename T, bool FWD, int NC = 6, int NA = Plan<N>::N1, int TV = 0>
__global__ void __launch_bounds__(Cfg<N, T, NA, TV>::T2) k_p24(PassArgs a) {
    using C = Cfg<N, T, NA, TV>;
    constexpr int H = C::H, W = C::W2, S = C::S2, NT = C::T2;
    constexpr int N1 = NA, N2 = N / NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [S][N][W]
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    if (a.cg && a.cg[f].done) return;
    const int tid = threadIdx.x;
    if (a.red_in && blockIdx.x == 0 && blockIdx.y == 0) {
        // alpha = <r, r> / <p, C : p> of the fused CG iteration, from the
        // block partials of P1 (thread t takes blocks t, t + NT, ...; then
        // a fixed tree), before this block's share of the transform
        const double* in = a.red_in + (size_t)f * a.red_n;
        double acc = 0.0;
        for (int b = tid; b < a.red_n; b += NT) acc += in[b];
        acc = block_sum_any(acc);
        if (tid == 0) cg_after_dot(a.cg + f, acc);
    }
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, slab0 = blockIdx.y * S;
    cplx<T>* sp = (cplx<T>*)a.out + f * a.sstride;
    constexpr int P = S * W;
    if (FWD) {
        for (int it = tid; it < P * N2; it += NT) {
            const int pc = it % P, t = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < NC * N)
                fwdA<N, N1, T>(sp + (long long)slab * N * H + col, H, buf + s * N * W + w, W, t, tw);
        }
        __syncthreads();
        for (int it = tid; it < P * N1; it += NT) {
            const int pc = it % P, k1 = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < NC * N)
                fwdB<N, N1, true, T>(buf + s * N * W + w, W, sp + (long long)slab * N * H + col, H, k1, tw);
        }
    } else {
        for (int it = tid; it < P * N1; it += NT) {
            const int pc = it % P, k1 = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < NC * N)
                invB<N, N1, true, T>(sp + (long long)slab * N * H + col, H, buf + s * N * W + w, W, k1, tw);
        }
        __syncthreads();
        for (int it = tid; it < P * N2; it += NT) {
            const int pc = it % P, t = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < NC * N)
                invA<N, N1, T>(buf + s * N * W + w, W, sp + (long long)slab * N * H + col, H, t, tw);
        }
    }
}

// 1/sqrt(x): CUDA's rsqrtf (about 2 ulp, far inside the FP32 path's
// tolerance) and rsqrt (1 ulp) in FP64.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// Ghat : tau at frequency (f1, f2, f3), times `scale`, in place on the six
// complex components (11, 22, 33, 23, 13, 12) held at stride `cs` in shared
// memory. With n = xi/|xi|, t = tau n and u = t - (n.t/2) n, the closed form
// n(x)t + t(x)n - (n.t) n(x)n equals n(x)u + u(x)n (Appendix A); at xi = 0
// the factor 1/|xi| is taken as 0, so the mean mode maps to zero.
template <typename T>
__device__ __forceinline__ void ghat_point(cplx<T>* b, int cs, int f1, int f2, int f3, T scale) {
    const T q2 = T(f1) * T(f1) + T(f2) * T(f2) + T(f3) * T(f3);
    const T inv = q2 > T(0) ? rsqrt_t(q2) : T(0);
    const T n0 = T(f1) * inv, n1 = T(f2) * inv, n2 = T(f3) * inv;
    cplx<T> c[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) c[k] = b[k * cs];
    const cplx<T> t0 = n0 * c[0] + n1 * c[5] + n2 * c[4];
    const cplx<T> t1 = n0 * c[5] + n1 * c[1] + n2 * c[3];
    const cplx<T> t2 = n0 * c[4] + n1 * c[3] + n2 * c[2];
    const cplx<T> h = signed_by<-1>(half_of(n0 * t0 + n1 * t1 + n2 * t2));  // -(n.t)/2, exactly
    const cplx<T> u0 = t0 + n0 * h, u1 = t1 + n1 * h, u2 = t2 + n2 * h;
    const T m0 = scale * n0, m1 = scale * n1, m2 = scale * n2;
    b[0 * cs] = (m0 + m0) * u0;  // 2 m, exactly
    b[1 * cs] = (m1 + m1) * u1;
    b[2 * cs] = (m2 + m2) * u2;
    b[3 * cs] = m1 * u2 + m2 * u1;
    b[4 * cs] = m0 * u2 + m2 * u0;
    b[5 * cs] = m0 * u1 + m1 * u0;
}

// ------------------------------------------------------------- P3 (x1 + Ghat)
// Stage A forward (global -> shared), stage B forward in place, Ghat with
// one thread per (column, frequency) holding all six components, stage B
// inverse in place, stage A inverse (shared -> global). Ghat as its own
// phase does each point once; fusing it into stage B's registers with the
// six components split over a lane pair duplicated n . tau n and needed
// shuffles (at 243^3 the separate phase took P3 from 0.206 to 0.185 ms in
// FP32 and from 7.4 to 6.2 ms in FP64).
//
// The middle of a tile (W columns of one x2 frequency, all six components,
// after stage A): stage B forward in place (permuted order), Ghat, stage B
// inverse in place; the caller synchronises before and after.
template <int N, int N1, int W, int NT, typename T>
__device__ __forceinline__ void p3_tile_middle(cplx<T>* buf, const cplx<T>* tw, int col0, int k2g, T scale,
                                               int tid) {
    constexpr int H = (N + 1) / 2, N2 = N / N1, P = 6 * W;
    const int f2 = (k2g <= (N - 1) / 2) ? k2g : k2g - N;
    if (N2 > 1) {
        for (int it = tid; it < P * N1; it += NT) {
            const int pc = it % P, k1 = it / P;
            const int c = pc / W, w = pc - c * W;
            if (col0 + w < H) fwdB<N, N1, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
        }
        __syncthreads();
    }
    for (int it = tid; it < W * N; it += NT) {
        const int w = it % W, pos = it / W, col = col0 + w;
        const int k1 = pos / N2, k2 = pos - k1 * N2;
        const int kk = k1 + N1 * k2;  // frequency held at position N2*k1 + k2
        if (col < H) ghat_point<T>(buf + pos * W + w, N * W, (kk <= (N - 1) / 2) ? kk : kk - N, f2, col, scale);
    }
    __syncthreads();
    if (N2 > 1) {
        for (int it = tid; it < P * N1; it += NT) {
            const int pc = it % P, k1 = it / P;
            const int c = pc / W, w = pc - c * W;
            if (col0 + w < H) invB<N, N1, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
        }
    }
}

template <int N, typename T, int NA = Plan<N>::N1, int TV = 0>
__global__ void __launch_bounds__(Cfg<N, T, NA, TV>::T3, (sizeof(T) == 4 && Cfg<N, T, NA, TV>::T3 <= 512)
                                                      ? (Cfg<N, T, NA, TV>::T3 <= 256 ? 4 : 2)
                                                      : is_dd_v<T> ? FFTG_DD_P3_MINB : 1) k_p3(PassArgs a) {
    using C = Cfg<N, T, NA, TV>;
    constexpr int H = C::H, W = C::W3, NT = C::T3;
    constexpr int N1 = NA, N2 = N / NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [6][N][W]
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    if (a.cg && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, k2g = blockIdx.y;
    cplx<T>* sp = (cplx<T>*)a.out + f * a.sstride;
    constexpr int P = 6 * W;
    const long long NH = (long long)N * H;
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) fwdA<N, N1, T>(sp + c * N * NH + k2g * H + col, (int)NH, buf + c * N * W + w, W, t, tw);
    }
    __syncthreads();
    p3_tile_middle<N, N1, W, NT, T>(buf, tw, col0, k2g, (T)a.scale, tid);
    __syncthreads();
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) invA<N, N1, T>(buf + c * N * W + w, W, sp + c * N * NH + k2g * H + col, (int)NH, t, tw);
    }
}

// P3 with stage B, Ghat and the inverse stage B in one phase (FP32, two-stage
// splits with N2 <= 9). One thread per (column, k1) streams the six
// components through its N2-point forward DFT and accumulates, for its N2
// frequencies kk = k1 + N1 k2, only t = tau n: the closed form of Ghat
// (Appendix A) needs tau through t alone, as n(x)u + u(x)n with
// u = t - (n.t / 2) n. Each output component is then formed from n and u,
// taken through the inverse N2-point DFT with its twiddles, and stored back
// in place. Against the default tile this passes each point through shared
// memory twice instead of five times and needs two barriers instead of
// four, at up to 128 registers per thread (blocks of at most 256 threads,
// two per SM). The results agree with the default's to FP32 rounding (t is
// summed in another order).
template <int N, int NA>
struct P3f {
    using C = Cfg<N, float, NA, 0>;
    static constexpr int W = C::W3, N1 = NA, N2 = N / NA;
    static constexpr bool ok = N2 > 1 && N2 <= 9;
    static constexpr int rup32(int x) { return ((x + 31) / 32) * 32; }
    // stage-A items in two rounds and one thread per fused item, within 256
    // threads (two blocks per SM at up to 128 registers each)
    static constexpr int TA0 = rup32((6 * W * N2 + 1) / 2), TB0 = rup32(W * N1);
    static constexpr int TA = TA0 > 256 ? 256 : TA0, TB = TB0 > 256 ? 256 : TB0;
    static constexpr int NT = TA > TB ? TA : TB;
};

template <int N, int NA>
__global__ void __launch_bounds__(P3f<N, NA>::NT, 2) k_p3f(PassArgs a) {
    using T = float;
    using S = P3f<N, NA>;
    static_assert(S::ok, "fused P3 needs a two-stage split with N2 <= 9");
    constexpr int H = (N + 1) / 2, W = S::W, N1 = NA, N2 = N / NA, NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [6][N][W]
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    if (a.cg && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, k2g = blockIdx.y;
    cplx<T>* sp = (cplx<T>*)a.out + f * a.sstride;
    constexpr int P = 6 * W;
    const long long NH = (long long)N * H;
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) fwdA<N, N1, T>(sp + c * N * NH + k2g * H + col, (int)NH, buf + c * N * W + w, W, t, tw);
    }
    __syncthreads();
    const T scale = (T)a.scale;
    const T f2 = (T)((k2g <= (N - 1) / 2) ? k2g : k2g - N);
    for (int it = tid; it < W * N1; it += NT) {
        const int w = it % W, k1 = it / W, col = col0 + w;
        if (col >= H) continue;
        cplx<T>* base = buf + (N2 * k1) * W + w;  // position N2*k1 + q at base[q * W]
        T n[N2][3];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int kk = k1 + N1 * k2;
            const T f1 = (T)((kk <= (N - 1) / 2) ? kk : kk - N), f3 = (T)col;
            const T q2 = f1 * f1 + f2 * f2 + f3 * f3;
            const T inv = q2 > T(0) ? rsqrt_t(q2) : T(0);
            n[k2][0] = f1 * inv;
            n[k2][1] = f2 * inv;
            n[k2][2] = f3 * inv;
        }
        cplx<T> t[N2][3];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) t[k2][0] = t[k2][1] = t[k2][2] = mk(T(0), T(0));
        // t = tau n over the components (11, 22, 33, 23, 13, 12)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            cplx<T> v[N2];
#pragma unroll
            for (int q = 0; q < N2; ++q) v[q] = base[c * N * W + q * W];
            RegDFT<N, N2, -1, T>::run(v, tw);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                if (c < 3) {
                    t[k2][c] = t[k2][c] + n[k2][c] * v[k2];
                } else {
                    // off-diagonal (i, j): 23 -> (1, 2), 13 -> (0, 2), 12 -> (0, 1)
                    const int i = c == 3 ? 1 : 0, j = c == 5 ? 1 : 2;
                    t[k2][i] = t[k2][i] + n[k2][j] * v[k2];
                    t[k2][j] = t[k2][j] + n[k2][i] * v[k2];
                }
            }
        }
        // u = t - (n.t / 2) n, in place
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const cplx<T> h = T(-0.5) * (n[k2][0] * t[k2][0] + n[k2][1] * t[k2][1] + n[k2][2] * t[k2][2]);
#pragma unroll
            for (int i = 0; i < 3; ++i) t[k2][i] = t[k2][i] + n[k2][i] * h;
        }
        // each output component: scale (n(x)u + u(x)n), inverse DFT, twiddle, store
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            cplx<T> v[N2];
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                if (c < 3) {
                    v[k2] = (T(2) * scale * n[k2][c]) * t[k2][c];
                } else {
                    const int i = c == 3 ? 1 : 0, j = c == 5 ? 1 : 2;
                    v[k2] = (scale * n[k2][i]) * t[k2][j] + (scale * n[k2][j]) * t[k2][i];
                }
            }
            RegDFT<N, N2, +1, T>::run(v, tw);
#pragma unroll
            for (int q = 0; q < N2; ++q) {
                cplx<T> z = v[q];
                if (k1 > 0 && q > 0) z = twmul<+1>(z, tw[q * k1]);  // q*k1 < N
                base[c * N * W + q * W] = z;
            }
        }
    }
    __syncthreads();
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) invA<N, N1, T>(buf + c * N * W + w, W, sp + c * N * NH + k2g * H + col, (int)NH, t, tw);
    }
}

// ----------------------------------------------------------------------- P5
// T: FFT precision; TO: output real type (P5_RHS writes the CG residual r
// in the inner precision).
template <int N, typename T, int MODE, typename TO, int NA = Plan<N>::N1, int TV = 0>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? FFTG_P5_MINB : is_dd_v<T> ? FFTG_DD_MINB : 2)
    k_p5(PassArgs a) {
    using C = Cfg<N, T, NA, TV>;
    constexpr int R = C::R, H = C::H;
    constexpr int N1 = NA, N2 = N / NA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [3][R][N]
    const int f = blockIdx.z;
    CGState* cg = a.cg ? a.cg + f : nullptr;
    if (a.active && !a.active[f]) return;
    if ((MODE == P5_DOT || MODE == P5_CGF) && cg->done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const cplx<T>* in = (const cplx<T>*)a.in + f * a.sstride;
    const long long HS = (long long)N * N * H;
    // Spectrum rows -> tile: the loads of FFTG_P5_LDB rounds are issued
    // before their stores, so that more of them are in flight.
    constexpr int NRL = (R * H + kThreads - 1) / kThreads;
    constexpr int LB = FFTG_P5_LDB < NRL ? FFTG_P5_LDB : NRL;
#pragma unroll
    for (int r0 = 0; r0 < NRL; r0 += LB) {
        cplx<T> A[LB][3], B[LB][3];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int it = tid + (r0 + u) * kThreads;
            if (r0 + u < NRL && it < nrows * H) {
                const int row = it / H, k = it - row * H;
                const long long o = (long long)(row0 + row) * H + k;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    A[u][c] = in[(2 * c) * HS + o];
                    B[u][c] = in[(2 * c + 1) * HS + o];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int it = tid + (r0 + u) * kThreads;
            if (r0 + u < NRL && it < nrows * H) {
                const int row = it / H, k = it - row * H;
                const int pk = perm_pos<N, N1>(k);
                const int pn = perm_pos<N, N1>(k == 0 ? 0 : N - k);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const cplx<T> a0 = A[u][c], b0 = B[u][c];
                    z[(c * R + row) * N + pk] = mk(a0.x - b0.y, a0.y + b0.x);  // A + iB
                    if (k > 0) z[(c * R + row) * N + pn] = mk(a0.x + b0.y, b0.x - a0.y);  // conj(A) + i conj(B)
                }
            }
        }
    }
    __syncthreads();
    constexpr int NP = 3 * R;
    if (N2 > 1) {
        for (int it = tid; it < NP * N1; it += kThreads) {
            const int pc = it % NP, k1 = it / NP;
            if (pc % R < nrows) invB<N, N1, false, T>(z + pc * N, 1, z + pc * N, 1, k1, tw);
        }
        __syncthreads();
    }
    for (int it = tid; it < NP * N2; it += kThreads) {
        const int pc = it % NP, t = it / NP;
        if (pc % R < nrows) invA<N, N1, T>(z + pc * N, 1, z + pc * N, 1, t, tw);
    }
    __syncthreads();
    const long long cs = a.cs;
    TO* out = (TO*)a.out + f * a.fstride;
    T acc0 = T(0);
    double acc1 = 0.0;
    // VO voxels per lane (FFTG_P5_VW, at most 16 bytes of TO): one vector
    // per component for q and p. With VO = 1 the tile reads are free of bank
    // conflicts. Lanes past the grid in the last block write only component
    // padding and are left out of the sums.
    constexpr int VO = (FFTG_P5_VW * (int)sizeof(TO) > 16) ? 16 / (int)sizeof(TO) : FFTG_P5_VW;
    // FFTG_P5_PB rounds at a time: the loads of p for all of them first.
    constexpr int NV = (R * N) / VO;
    constexpr int NRE = (NV + kThreads - 1) / kThreads;
    constexpr int PB = FFTG_P5_PB < NRE ? FFTG_P5_PB : NRE;
    // P5_DOT: p; P5_CGF: r (updated in place, r -= alpha q)
    const TO* pin = (const TO*)a.aux + f * a.fstride;
    TO* rout = MODE == P5_CGF ? (TO*)a.aux3 + f * a.fstride : nullptr;
    const TO alpha = MODE == P5_CGF ? (TO)cg->alpha : TO(0);
#pragma unroll
    for (int r0 = 0; r0 < NRE; r0 += PB) {
        TO pv[PB][6][VO];
        if (MODE == P5_DOT || MODE == P5_CGF) {
#pragma unroll
            for (int u = 0; u < PB; ++u) {
                const int j = tid + (r0 + u) * kThreads;
                if (r0 + u < NRE && j < NV && j * VO < nel) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) ldv<VO, TO>(pin + c * cs + base + j * VO, pv[u][c]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            const int j = tid + (r0 + u) * kThreads;
            const int i0 = j * VO;
            if (!(r0 + u < NRE && j < NV && i0 < nel)) continue;
            const long long v0 = base + i0;
            TO q[6][VO];
            T qd[6][VO];
#pragma unroll
            for (int e = 0; e < VO; ++e) {
                const cplx<T> z0 = z[i0 + e], z1 = z[R * N + i0 + e], z2 = z[2 * R * N + i0 + e];
                qd[0][e] = z0.x;
                qd[1][e] = z0.y;
                qd[2][e] = z1.x;
                qd[3][e] = z1.y;
                qd[4][e] = z2.x;
                qd[5][e] = z2.y;
#pragma unroll
                for (int c = 0; c < 6; ++c) q[c][e] = (TO)qd[c][e];
            }
            if (MODE == P5_CGF) {
                // r -= alpha q, <r, r> (lanes past the grid update padding only)
#pragma unroll
                for (int c = 0; c < 6; ++c) {
#pragma unroll
                    for (int e = 0; e < VO; ++e) pv[u][c][e] -= alpha * q[c][e];
                    stv<VO, TO>(rout + c * cs + v0, pv[u][c]);
                }
#pragma unroll
                for (int e = 0; e < VO; ++e) {
                    if (i0 + e < nel) {
                        const TO re[6] = {pv[u][0][e], pv[u][1][e], pv[u][2][e], pv[u][3][e], pv[u][4][e], pv[u][5][e]};
                        acc0 += (T)frob<TO>(re, re);
                    }
                }
                continue;
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) stv<VO, TO>(out + c * cs + v0, q[c]);
            if (MODE == P5_DOT) {
#pragma unroll
                for (int e = 0; e < VO; ++e) {
                    if (i0 + e < nel) {
                        const TO pe[6] = {pv[u][0][e], pv[u][1][e], pv[u][2][e], pv[u][3][e], pv[u][4][e], pv[u][5][e]};
                        const TO qe[6] = {q[0][e], q[1][e], q[2][e], q[3][e], q[4][e], q[5][e]};
                        acc0 += (T)frob<TO>(pe, qe);
                    }
                }
            } else if (MODE == P5_RHS) {
#pragma unroll
                for (int e = 0; e < VO; ++e) {
                    if (i0 + e < nel) {
                        const T qde[6] = {qd[0][e], qd[1][e], qd[2][e], qd[3][e], qd[4][e], qd[5][e]};
                        const TO qe[6] = {q[0][e], q[1][e], q[2][e], q[3][e], q[4][e], q[5][e]};
                        acc1 += (double)frob<T>(qde, qde);
                        acc0 += (T)frob<TO>(qe, qe);
                    }
                }
            }
        }
    }
    if (MODE == P5_PLAIN) return;
    const int nb = gridDim.x;
    double part[2];
    part[0] = block_sum((double)acc0);
    if (MODE == P5_CGF) {
        // the block's part of <r, r>; k_cg_rr reduces the parts (no fence
        // or ticket at the end of every block here)
        if (tid == 0) a.partials[(size_t)f * nb + blockIdx.x] = part[0];
        return;
    }
    part[1] = (MODE == P5_RHS) ? block_sum(acc1) : 0.0;
    double* partials = a.partials + (size_t)f * nb * 2;
    if (!publish_partials<2>(part, partials, blockIdx.x, nb, &cg->ticket)) return;
    double tot[2];
    reduce_partials<2>(partials, nb, &cg->ticket, tot);
    if (tid != 0) return;
    if (MODE == P5_DOT)
        cg_after_dot(cg, tot[0]);
    else
        cg_start(cg, tot[0], tot[1]);
}

// ------------------------------------------------------------------ launcher
enum PassKind : int {
    PK_P1_PLAIN_F64, PK_P1_PLAIN_F32, PK_P1_TAN_F64, PK_P1_TAN_F32, PK_P1_CG_F64, PK_P1_CG_F32,
    PK_P1_TANRHS_F64, PK_P1_TANRHS_F32,
    PK_P2_F64, PK_P2_F32, PK_P4_F64, PK_P4_F32, PK_P3_F64, PK_P3_F32,
    PK_P5_PLAIN_F64, PK_P5_PLAIN_F32, PK_P5_DOT_F64, PK_P5_DOT_F32,
    PK_P5_RHS_F64_TO_F64, PK_P5_RHS_F64_TO_F32, PK_P5_RHS_F32_TO_F32,
    // double-float FFTs (the mixed path's residual): FP64 field in, FP32
    // residual or FP64 field out
    PK_P1_PLAIN_DD, PK_P2_DD, PK_P3_DD, PK_P4_DD, PK_P5_RHS_DD_TO_F32, PK_P5_PLAIN_DD_TO_F64,
    // the CG iteration without the update pass (P1_CGF / P5_CGF), FP32
    PK_P1_CGF_F32, PK_P5_CGF_F32,
    PK_COUNT
};

// Grid geometry of the row passes (blocks per field): needed by the host to
// size the partial-sum buffer.
int row_blocks(int N, bool fp64);

cudaError_t run_pass(int N, PassKind kind, const PassArgs& a, int nf, cudaStream_t s);

template <int N>
cudaError_t run_pass_n(PassKind kind, const PassArgs& a, int nf, cudaStream_t s);

template <typename K>
static cudaError_t launch_k(K kernel, dim3 grid, size_t smem, const PassArgs& a, cudaStream_t s,
                            int threads = kThreads) {
    static_assert(sizeof(PassArgs) < 4096, "kernel params");
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t run_pass_n(PassKind kind, const PassArgs& a, int nf, cudaStream_t s) {
    using C32 = Cfg<N, float>;
    using C64 = Cfg<N, double>;
    using CDD = Cfg<N, dd>;
    static_assert(CDD::row_blocks == C64::row_blocks && CDD::W2 == C64::W2 && CDD::S2 == C64::S2,
                  "double-float row and column passes share the FP64 geometry");
    const dim3 r32(C32::row_blocks, 1, nf), r64(C64::row_blocks, 1, nf);
    const dim3 c32((C32::H + C32::W2 - 1) / C32::W2, (6 * N + C32::S2 - 1) / C32::S2, nf);
    const dim3 c64((C64::H + C64::W2 - 1) / C64::W2, (6 * N + C64::S2 - 1) / C64::S2, nf);
    const dim3 g32((C32::H + C32::W3 - 1) / C32::W3, N, nf);
    const dim3 g64((C64::H + C64::W3 - 1) / C64::W3, N, nf);
    const dim3 gdd((CDD::H + CDD::W3 - 1) / CDD::W3, N, nf);
    switch (kind) {
        case PK_P1_PLAIN_F64: return launch_k(k_p1<N, double, P1_PLAIN>, r64, C64::smem_rows, a, s);
        case PK_P1_PLAIN_F32: return launch_k(k_p1<N, float, P1_PLAIN>, r32, C32::smem_rows, a, s);
        case PK_P1_TAN_F64: return launch_k(k_p1<N, double, P1_TAN>, r64, C64::smem_rows, a, s);
        case PK_P1_TAN_F32: return launch_k(k_p1<N, float, P1_TAN>, r32, C32::smem_rows, a, s);
        case PK_P1_CG_F64: return launch_k(k_p1<N, double, P1_CG>, r64, C64::smem_rows, a, s);
        case PK_P1_CG_F32: return launch_k(k_p1<N, float, P1_CG>, r32, C32::smem_rows, a, s);
        case PK_P1_TANRHS_F64: return launch_k(k_p1<N, double, P1_TANRHS>, r64, C64::smem_rows, a, s);
        case PK_P1_TANRHS_F32: return launch_k(k_p1<N, float, P1_TANRHS>, r32, C32::smem_rows, a, s);
        case PK_P2_F64: return launch_k(k_p24<N, double, true>, c64, C64::smem_p24, a, s, C64::T2);
        case PK_P2_F32: return launch_k(k_p24<N, float, true>, c32, C32::smem_p24, a, s, C32::T2);
        case PK_P4_F64: return launch_k(k_p24<N, double, false>, c64, C64::smem_p24, a, s, C64::T2);
        case PK_P4_F32: return launch_k(k_p24<N, float, false>, c32, C32::smem_p24, a, s, C32::T2);
        case PK_P3_F64: return launch_k(k_p3<N, double>, g64, C64::smem_p3, a, s, C64::T3);
        case PK_P3_F32: return launch_k(k_p3<N, float>, g32, C32::smem_p3, a, s, C32::T3);
        case PK_P5_PLAIN_F64: return launch_k(k_p5<N, double, P5_PLAIN, double>, r64, C64::smem_rows, a, s);
        case PK_P5_PLAIN_F32: return launch_k(k_p5<N, float, P5_PLAIN, float>, r32, C32::smem_rows, a, s);
        case PK_P5_DOT_F64: return launch_k(k_p5<N, double, P5_DOT, double>, r64, C64::smem_rows, a, s);
        case PK_P5_DOT_F32: return launch_k(k_p5<N, float, P5_DOT, float>, r32, C32::smem_rows, a, s);
        case PK_P5_RHS_F64_TO_F64:
            return launch_k(k_p5<N, double, P5_RHS, double>, r64, C64::smem_rows, a, s);
        case PK_P5_RHS_F64_TO_F32:
            return launch_k(k_p5<N, double, P5_RHS, float>, r64, C64::smem_rows, a, s);
        case PK_P5_RHS_F32_TO_F32:
            return launch_k(k_p5<N, float, P5_RHS, float>, r32, C32::smem_rows, a, s);
        case PK_P1_PLAIN_DD: return launch_k(k_p1<N, dd, P1_PLAIN>, r64, CDD::smem_rows, a, s);
        case PK_P2_DD: return launch_k(k_p24<N, dd, true>, c64, CDD::smem_p24, a, s, CDD::T2);
        case PK_P4_DD: return launch_k(k_p24<N, dd, false>, c64, CDD::smem_p24, a, s, CDD::T2);
        case PK_P3_DD: return launch_k(k_p3<N, dd>, gdd, CDD::smem_p3, a, s, CDD::T3);
        case PK_P5_RHS_DD_TO_F32: return launch_k(k_p5<N, dd, P5_RHS, float>, r64, CDD::smem_rows, a, s);
        case PK_P5_PLAIN_DD_TO_F64:
            return launch_k(k_p5<N, dd, P5_PLAIN, double>, r64, CDD::smem_rows, a, s);
        case PK_P1_CGF_F32: return launch_k(k_p1<N, float, P1_CGF>, r32, C32::smem_rows, a, s);
        case PK_P5_CGF_F32: return launch_k(k_p5<N, float, P5_CGF, float>, r32, C32::smem_rows, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftg
