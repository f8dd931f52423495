// Grid passes of the finite-strain extension (Section 6 names finite strain
// as the next step of the method): the projected matvec q = G (K : p) and
// the residual G P on real fields of nine components, the deformation-
// gradient-like tensor A_ij at component 3i + j, [9][cs], and a half
// spectrum [9][N][N][H].
//
// The five passes are those of the small-strain path with three changes:
//  * nine real components share five complex FFTs per row (pairs (0,1),
//    (2,3), (4,5), (6,7) and component 8 alone);
//  * the projection onto gradient fields acts row by row: with n = xi/|xi|,
//    Ghat : A = (A n) (x) n, i.e. Ghat_ijlm = delta_il n_j n_m (the
//    finite-strain counterpart of Appendix A's operator; Ghat(0) = 0);
//  * the tangent is St. Venant-Kirchhoff's, applied on the fly from the
//    displacement gradient H = F - I (the only per-voxel tangent data) and
//    the phase's Lame constants: K : d = d S + F dS with
//    E = (H + H^T + H^T H)/2, S = lambda tr(E) I + 2 mu E, M = F^T d and
//    dS = lambda tr(M) I + mu (M + M^T).
// The mixed path's residual runs the plain passes in double-float
// arithmetic (dd.cuh) on the FP64 stress.
#pragma once

#include "common.cuh"
#include "fft_core.cuh"
#include "passes.cuh"

namespace fftg {

constexpr int kFsComp = 9;
constexpr int kFsPairs = 5;

enum : int { FS_P1_PLAIN = 0, FS_P1_TAN = 1, FS_P1_CG = 2, FS_P1_TANRHS = 3, FS_P1_CGF = 4 };
enum : int { FS_P5_PLAIN = 0, FS_P5_DOT = 1, FS_P5_RHS = 2, FS_P5_CGF = 3 };
// FS_P1_CGF / FS_P5_CGF: the CG iteration without the update pass, as in
// the small-strain passes (P1_CGF): G projects orthogonally onto gradient
// fields, so <p, G K p> = <p, K p> for a gradient field p; P1 reduces
// <p, K : p> (alpha), P5 updates r -= alpha q and reduces <r, r>.

struct FsArgs {
    const void* in;        // P1: real field; P5: spectrum
    void* out;             // P1: spectrum; P2-P4: spectrum (in place); P5: real field
    const void* aux;       // P1_CG: r; P5_DOT: p
    void* aux2;            // P1_CG: p (updated in place)
    void* aux3;            // P1_CG: x (gets the previous iteration's alpha p)
    const void* hgrad;     // P1_TAN, P1_CG: H = F - I, [9][cs] in the FFT precision
    const uint8_t* phase;  // [cs]
    const double* lame;    // [nphase][2]: lambda, mu
    CGState* cg;
    double* partials;      // [row blocks][2]
    const void* tw;        // w_N^j, j < N, in the FFT precision
    double scale;          // P3: factor on Ghat (+-1/N^3)
    long long cs;          // component stride of the real fields (elements)
    int unit;              // P1_TANRHS: tau = K : E_unit, E_unit the unit tensor at component unit
    const double* red_in;  // P2 of the fused CG iteration: P1's block partials of <p, K : p>
    int red_n;             // (reduced by P2's first block, which sets alpha)
};

// Tuning: voxels per lane in the elementwise phases of P1 and P5 (moved as
// one vector per component; FP64 at most 2), shared-memory budgets (KB) of
// the row passes and of P3, and the minimum resident blocks per SM of the
// FP32 P1 and P5 (a bound on their registers; the FP64 ones take what they
// need: they are bound by FP64 arithmetic, not by memory). Set by timing
// variants on the 243^3 finite-strain workload (per CG iteration, FP32):
// one voxel per lane and 40 KB of rows (R = 4) gave P1 0.66 ms (3 or 4
// blocks per SM alike; 4 spills a little) and P5 0.34 ms with 4 blocks per
// SM (0.39 ms with 3); two voxels per lane 0.73-0.91 ms for P1 (it spills
// at 3 blocks per SM); 80 KB of rows 0.76 ms; P3 with 100 or 64 KB of
// columns 0.44 and 0.71 ms against 0.39 ms with 150 KB. P5 with the
// spectrum loads of two rounds issued together: 0.323 against 0.336 ms
// (with 3 blocks per SM 0.369 ms).
#ifndef FFTG_FS_VW
#define FFTG_FS_VW 1
#endif
#ifndef FFTG_FS_ROW_KB
#define FFTG_FS_ROW_KB 40
#endif
#ifndef FFTG_FS_P3_KB
#define FFTG_FS_P3_KB 150
#endif
#ifndef FFTG_FS_P1_MINB
#define FFTG_FS_P1_MINB 3
#endif
#ifndef FFTG_FS_P5_MINB
#define FFTG_FS_P5_MINB 4
#endif
#ifndef FFTG_FS_P5_LDB
#define FFTG_FS_P5_LDB 2
#endif

template <int N, typename T>
struct FsCfg {
    static constexpr int H = (N + 1) / 2;
    static constexpr int CS = (int)sizeof(cplx<T>);
    static constexpr int fl2(int x) {
        return x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1;
    }
    static constexpr int rup32(int x) { return ((x + 31) / 32) * 32; }
    static constexpr int cap(int x) { return x > 1024 ? 1024 : x; }
    // rows per block of P1/P5: five complex pencils per row; a power of two
    // >= 4, so a block's rows start on a 16-byte boundary of every component
    static constexpr int R0 = fl2(FFTG_FS_ROW_KB * 1024 / (kFsPairs * N * CS));
    static constexpr int R = R0 < 4 ? 4 : R0;
    static constexpr int VW = (sizeof(T) == 8 && FFTG_FS_VW > 2) ? 2 : FFTG_FS_VW;
    // columns per block of P3: nine pencils per column
    static constexpr int W3 = fl2(FFTG_FS_P3_KB * 1024 / (kFsComp * N * CS));
    static constexpr int T3 = Plan<N>::N2 == 1 ? 256 : cap(rup32(kFsComp * W3 * Plan<N>::N2));
    static constexpr size_t smem_rows = (size_t)(kFsPairs * R * N + N) * CS;
    static constexpr size_t smem_p3 = (size_t)(kFsComp * W3 * N + N) * CS;
    static constexpr int row_blocks = (N * N + R - 1) / R;
    static_assert(smem_rows <= 227 * 1024 && smem_p3 <= 227 * 1024, "shared memory per block");
    static_assert(T3 <= 1024 && T3 % 32 == 0, "threads per block");
    static_assert((R * N) % VW == 0 && (VW == 1 || VW == 2 || VW == 4), "vector width");
};

// tau = K(F) : d for St. Venant-Kirchhoff, from h = F - I.
template <typename T>
__device__ __forceinline__ void svk_tangent_apply(const T (&h)[9], T lam, T mu, const T (&d)[9], T (&tau)[9]) {
    T E[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T hh = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) hh += h[3 * k + i] * h[3 * k + j];
            E[3 * i + j] = T(0.5) * (h[3 * i + j] + h[3 * j + i] + hh);
        }
    const T le = lam * (E[0] + E[4] + E[8]);
    T M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T m = d[3 * i + j];  // (I + H)^T d
#pragma unroll
            for (int k = 0; k < 3; ++k) m += h[3 * k + i] * d[3 * k + j];
            M[3 * i + j] = m;
        }
    const T lm = lam * (M[0] + M[4] + M[8]);
    T S[9], dS[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S[3 * i + j] = T(2) * mu * E[3 * i + j] + (i == j ? le : T(0));
            dS[3 * i + j] = mu * (M[3 * i + j] + M[3 * j + i]) + (i == j ? lm : T(0));
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T t = dS[3 * i + j];  // I dS
#pragma unroll
            for (int k = 0; k < 3; ++k) t += d[3 * i + k] * S[3 * k + j] + h[3 * i + k] * dS[3 * k + j];
            tau[3 * i + j] = t;
        }
}

// ----------------------------------------------------------------------- P1
// [x += alpha p; p = r + beta p]; tau = K : p or tau = input; x3 R2C FFT of
// R rows per block.
template <int N, typename T, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? FFTG_FS_P1_MINB : 1) k_fs_p1(FsArgs a) {
    using C = FsCfg<N, T>;
    constexpr int R = C::R, H = C::H, VW = C::VW;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [5][R][N]
    constexpr bool CGM = MODE == FS_P1_CG || MODE == FS_P1_CGF;
    if (CGM && a.cg->done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const long long cs = a.cs;
    T beta = T(0), alpha = T(0);
    T pkp = T(0);  // FS_P1_CGF: this thread's part of <p, K : p>
    bool first = true;
    if (CGM) {
        beta = (T)a.cg->beta;
        alpha = (T)a.cg->alpha;
        first = a.cg->it == 0;
    }
    // Elementwise phase: VW consecutive voxels per lane, one vector per
    // component. Every load of an item is issued before its first store
    // (the fields could alias as far as the compiler knows, which would
    // otherwise serialise one round trip per component). In the last block
    // a vector that straddles the end of the grid touches only the padding
    // of each component (cs >= N^3 + 4), and its lanes past the grid belong
    // to rows the FFT stages skip.
    for (int j = tid; j < (R * N) / VW; j += kThreads) {
        const int i0 = j * VW;
        T s[9][VW];
        if (i0 < nel) {
            const long long v0 = base + i0;
            T p[9][VW], h[9][VW];
            int ph[VW];
            if (CGM) {
                const T* r = (const T*)a.aux;
                T* pp = (T*)a.aux2;
                T* xx = (T*)a.aux3;
                T po[9][VW], xo[9][VW];
#pragma unroll
                for (int c = 0; c < 9; ++c) ldv<VW, T>(r + c * cs + v0, p[c]);
                if (!first) {
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        ldv<VW, T>(pp + c * cs + v0, po[c]);
                        ldv<VW, T>(xx + c * cs + v0, xo[c]);
                    }
                }
                const T* hg = (const T*)a.hgrad;
#pragma unroll
                for (int c = 0; c < 9; ++c) ldv<VW, T>(hg + c * cs + v0, h[c]);
#pragma unroll
                for (int e = 0; e < VW; ++e) ph[e] = a.phase[v0 + e];
                if (!first) {
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
#pragma unroll
                        for (int e = 0; e < VW; ++e) {
                            xo[c][e] += alpha * po[c][e];
                            p[c][e] += beta * po[c][e];
                        }
                        stv<VW, T>(xx + c * cs + v0, xo[c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < 9; ++c) stv<VW, T>(pp + c * cs + v0, p[c]);
            } else {
                using TIn = typename PlainIn<T>::type;
                const TIn* in = (const TIn*)a.in;
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    TIn t[VW];
                    if (MODE == FS_P1_TANRHS) {
#pragma unroll
                        for (int e = 0; e < VW; ++e) t[e] = TIn(c == a.unit ? 1 : 0);
                    } else {
                        ldv<VW, TIn>(in + c * cs + v0, t);
                    }
#pragma unroll
                    for (int e = 0; e < VW; ++e) p[c][e] = T(t[e]);
                }
                if (MODE == FS_P1_TAN || MODE == FS_P1_TANRHS) {
                    const T* hg = (const T*)a.hgrad;
#pragma unroll
                    for (int c = 0; c < 9; ++c) ldv<VW, T>(hg + c * cs + v0, h[c]);
#pragma unroll
                    for (int e = 0; e < VW; ++e) ph[e] = a.phase[v0 + e];
                }
            }
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                if (MODE == FS_P1_PLAIN) {
#pragma unroll
                    for (int c = 0; c < 9; ++c) s[c][e] = p[c][e];
                } else {
                    T he[9], pe[9], se[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        he[c] = h[c][e];
                        pe[c] = p[c][e];
                    }
                    const double* m = a.lame + 2 * ph[e];
                    svk_tangent_apply<T>(he, (T)m[0], (T)m[1], pe, se);
#pragma unroll
                    for (int c = 0; c < 9; ++c) s[c][e] = se[c];
                    if (MODE == FS_P1_CGF && i0 + e < nel) {
#pragma unroll
                        for (int c = 0; c < 9; ++c) pkp += pe[c] * se[c];
                    }
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < 9; ++c)
#pragma unroll
                for (int e = 0; e < VW; ++e) s[c][e] = T(0);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
#pragma unroll
            for (int c = 0; c < 4; ++c) z[c * R * N + i0 + e] = mk(s[2 * c][e], s[2 * c + 1][e]);
            z[4 * R * N + i0 + e] = mk(s[8][e], T(0));
        }
    }
    // FS_P1_CGF: this block's part of <p, K : p> (P2 reduces the parts)
    __shared__ double pkp_warp[kThreads / 32];
    if (MODE == FS_P1_CGF) {
        const double wv = warp_sum((double)pkp);
        if ((tid & 31) == 0) pkp_warp[tid >> 5] = wv;
    }
    __syncthreads();
    if (MODE == FS_P1_CGF && tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += pkp_warp[w];
        a.partials[blockIdx.x] = t;
    }
    constexpr int NP = kFsPairs * R;
    for (int it = tid; it < NP * N2; it += kThreads) {
        const int pc = it % NP, t = it / NP;
        if (pc % R < nrows) fwdA<N, T>(z + pc * N, 1, z + pc * N, 1, t, tw);
    }
    __syncthreads();
    if (N2 > 1) {
        for (int it = tid; it < NP * N1; it += kThreads) {
            const int pc = it % NP, k1 = it / NP;
            if (pc % R < nrows) fwdB<N, false, T>(z + pc * N, 1, z + pc * N, 1, k1, tw);
        }
        __syncthreads();
    }
    // Split each packed transform Z = FFT(a + i b) into the half spectra
    // A_k = (Z_k + conj Z_{N-k})/2 and B_k = (Z_k - conj Z_{N-k})/(2i).
    cplx<T>* out = (cplx<T>*)a.out;
    const long long HS = (long long)N * N * H;
    for (int it = tid; it < nrows * H; it += kThreads) {
        const int row = it / H, k = it - row * H;
        const int pk = perm_pos<N>(k), pn = perm_pos<N>(k == 0 ? 0 : N - k);
        const long long o = (long long)(row0 + row) * H + k;
#pragma unroll
        for (int c = 0; c < kFsPairs; ++c) {
            const cplx<T> zk = z[(c * R + row) * N + pk];
            const cplx<T> zn = conj(z[(c * R + row) * N + pn]);
            out[(2 * c) * HS + o] = half_of(zk + zn);
            if (2 * c + 1 < kFsComp) {
                const cplx<T> d = zk - zn;
                out[(2 * c + 1) * HS + o] = half_of(mk(d.y, -d.x));
            }
        }
    }
}

// Ghat_fs : A at frequency (f1, f2, f3), times `scale`, in place on the nine
// complex components held at stride `cs`: row i becomes (A_i . n) n.
template <typename T>
__device__ __forceinline__ void ghat_fs_point(cplx<T>* b, int cs, int f1, int f2, int f3, T scale) {
    const T q2 = T(f1) * T(f1) + T(f2) * T(f2) + T(f3) * T(f3);
    const T inv = q2 > T(0) ? rsqrt_t(q2) : T(0);
    const T n0 = T(f1) * inv, n1 = T(f2) * inv, n2 = T(f3) * inv;
    const T m0 = scale * n0, m1 = scale * n1, m2 = scale * n2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const cplx<T> t = n0 * b[(3 * i) * cs] + n1 * b[(3 * i + 1) * cs] + n2 * b[(3 * i + 2) * cs];
        b[(3 * i) * cs] = m0 * t;
        b[(3 * i + 1) * cs] = m1 * t;
        b[(3 * i + 2) * cs] = m2 * t;
    }
}

// ------------------------------------------------------------- P3 (x1 + Ghat)
// As the small-strain P3: stage A forward into shared memory, stage B
// forward in place, Ghat_fs with one thread per (column, frequency), stage B
// inverse, stage A inverse back to the spectrum; in FP32 with two-stage
// splits of N2 <= 9 the middle three phases are one (below).
template <int N, typename T>
__global__ void __launch_bounds__(FsCfg<N, T>::T3) k_fs_p3(FsArgs a) {
    using C = FsCfg<N, T>;
    constexpr int H = C::H, W = C::W3, NT = C::T3;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [9][N][W]
    if (a.cg && a.cg->done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, k2g = blockIdx.y;
    cplx<T>* sp = (cplx<T>*)a.out;
    constexpr int P = kFsComp * W;
    const long long NH = (long long)N * H;
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) fwdA<N, T>(sp + c * N * NH + k2g * H + col, (int)NH, buf + c * N * W + w, W, t, tw);
    }
    __syncthreads();
    const T scale = (T)a.scale;
    const int f2 = (k2g <= (N - 1) / 2) ? k2g : k2g - N;
    if constexpr (std::is_same<T, float>::value && N2 > 1 && N2 <= 9) {
        // Stage B, Ghat_fs and the inverse stage B in one phase: row i of
        // Ghat_fs : A is (A_i . n) n, which needs row i's three components
        // only. One thread per (column, k1, row) takes them through the
        // forward N2-point DFT, sums t = A_i . n for its N2 frequencies in
        // Ghat_fs's order, and writes scale n_j t back through the inverse
        // DFT and its twiddles: two shared-memory passes per point instead
        // of five, and two barriers fewer.
        for (int it = tid; it < W * N1 * 3; it += NT) {
            const int w = it % W, r = it / W;
            const int k1 = r % N1, row = r / N1, col = col0 + w;
            if (col >= H) continue;
            cplx<T>* base = buf + (3 * row * N + N2 * k1) * W + w;  // component 3 row + j at base[j N W]
            T n[N2][3];
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int kk = k1 + N1 * k2;
                const T f1 = T((kk <= (N - 1) / 2) ? kk : kk - N), g2 = T(f2), f3 = T(col);
                const T q2 = f1 * f1 + g2 * g2 + f3 * f3;
                const T inv = q2 > T(0) ? rsqrt_t(q2) : T(0);
                n[k2][0] = f1 * inv;
                n[k2][1] = g2 * inv;
                n[k2][2] = f3 * inv;
            }
            cplx<T> t[N2];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cplx<T> v[N2];
#pragma unroll
                for (int q = 0; q < N2; ++q) v[q] = base[j * N * W + q * W];
                RegDFT<N, N2, -1, T>::run(v, tw);
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) t[k2] = j == 0 ? n[k2][0] * v[k2] : t[k2] + n[k2][j] * v[k2];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cplx<T> v[N2];
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) v[k2] = (scale * n[k2][j]) * t[k2];
                RegDFT<N, N2, +1, T>::run(v, tw);
#pragma unroll
                for (int q = 0; q < N2; ++q) {
                    cplx<T> z = v[q];
                    if (k1 > 0 && q > 0) z = twmul<+1>(z, tw[q * k1]);  // q*k1 < N
                    base[j * N * W + q * W] = z;
                }
            }
        }
    } else {
        if (N2 > 1) {
            for (int it = tid; it < P * N1; it += NT) {
                const int pc = it % P, k1 = it / P;
                const int c = pc / W, w = pc - c * W;
                if (col0 + w < H) fwdB<N, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
            }
            __syncthreads();
        }
        for (int it = tid; it < W * N; it += NT) {
            const int w = it % W, pos = it / W, col = col0 + w;
            const int k1 = pos / N2, k2 = pos - k1 * N2;
            const int kk = k1 + N1 * k2;  // frequency held at position N2*k1 + k2
            if (col < H)
                ghat_fs_point<T>(buf + pos * W + w, N * W, (kk <= (N - 1) / 2) ? kk : kk - N, f2, col, scale);
        }
        __syncthreads();
        if (N2 > 1) {
            for (int it = tid; it < P * N1; it += NT) {
                const int pc = it % P, k1 = it / P;
                const int c = pc / W, w = pc - c * W;
                if (col0 + w < H) invB<N, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
            }
        }
    }
    __syncthreads();
    for (int it = tid; it < P * N2; it += NT) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) invA<N, T>(buf + c * N * W + w, W, sp + c * N * NH + k2g * H + col, (int)NH, t, tw);
    }
}

// ----------------------------------------------------------------------- P5
// x3 C2R inverse FFT of R rows per block; writes the real field (in TO) and,
// for DOT, the partials of <p, q> (then alpha), for RHS those of <r, r> in
// TO and of ||G P||^2 in T (then the start of the CG solve).
template <int N, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? FFTG_FS_P5_MINB : 1) k_fs_p5(FsArgs a) {
    using C = FsCfg<N, T>;
    constexpr int R = C::R, H = C::H;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [5][R][N]
    CGState* cg = a.cg;
    if ((MODE == FS_P5_DOT || MODE == FS_P5_CGF) && cg->done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const cplx<T>* in = (const cplx<T>*)a.in;
    const long long HS = (long long)N * N * H;
    // Spectrum rows -> tile, the loads of FFTG_FS_P5_LDB rounds issued
    // before their stores.
    constexpr int NRL = (R * H + kThreads - 1) / kThreads;
    constexpr int LB = FFTG_FS_P5_LDB < NRL ? FFTG_FS_P5_LDB : NRL;
#pragma unroll
    for (int r0 = 0; r0 < NRL; r0 += LB) {
        cplx<T> A[LB][kFsPairs], B[LB][kFsPairs];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int it = tid + (r0 + u) * kThreads;
            if (r0 + u < NRL && it < nrows * H) {
                const int row = it / H, k = it - row * H;
                const long long o = (long long)(row0 + row) * H + k;
#pragma unroll
                for (int c = 0; c < kFsPairs; ++c) {
                    A[u][c] = in[(2 * c) * HS + o];
                    B[u][c] = (2 * c + 1 < kFsComp) ? in[(2 * c + 1) * HS + o] : mk(T(0), T(0));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int it = tid + (r0 + u) * kThreads;
            if (r0 + u < NRL && it < nrows * H) {
                const int row = it / H, k = it - row * H;
                const int pk = perm_pos<N>(k);
                const int pn = perm_pos<N>(k == 0 ? 0 : N - k);
#pragma unroll
                for (int c = 0; c < kFsPairs; ++c) {
                    const cplx<T> a0 = A[u][c], b0 = B[u][c];
                    z[(c * R + row) * N + pk] = mk(a0.x - b0.y, a0.y + b0.x);                  // A + iB
                    if (k > 0) z[(c * R + row) * N + pn] = mk(a0.x + b0.y, b0.x - a0.y);  // conj(A) + i conj(B)
                }
            }
        }
    }
    __syncthreads();
    constexpr int NP = kFsPairs * R;
    if (N2 > 1) {
        for (int it = tid; it < NP * N1; it += kThreads) {
            const int pc = it % NP, k1 = it / NP;
            if (pc % R < nrows) invB<N, false, T>(z + pc * N, 1, z + pc * N, 1, k1, tw);
        }
        __syncthreads();
    }
    for (int it = tid; it < NP * N2; it += kThreads) {
        const int pc = it % NP, t = it / NP;
        if (pc % R < nrows) invA<N, T>(z + pc * N, 1, z + pc * N, 1, t, tw);
    }
    __syncthreads();
    const long long cs = a.cs;
    TO* out = (TO*)a.out;
    const TO* pin = (const TO*)a.aux;   // FS_P5_DOT: p; FS_P5_CGF: r
    TO* rout = MODE == FS_P5_CGF ? (TO*)a.aux3 : nullptr;
    const TO alpha = MODE == FS_P5_CGF ? (TO)cg->alpha : TO(0);
    T acc0 = T(0);
    double acc1 = 0.0;
    // VO voxels per lane (at most 16 bytes of TO): p is loaded before q is
    // stored. Lanes past the grid in the last block write only component
    // padding and are left out of the sums.
    constexpr int VO = (C::VW * (int)sizeof(TO) > 16) ? 16 / (int)sizeof(TO) : C::VW;
    for (int j = tid; j < (R * N) / VO; j += kThreads) {
        const int i0 = j * VO;
        if (i0 >= nel) continue;
        const long long v0 = base + i0;
        TO pv[9][VO];
        if (MODE == FS_P5_DOT || MODE == FS_P5_CGF) {
#pragma unroll
            for (int c = 0; c < 9; ++c) ldv<VO, TO>(pin + c * cs + v0, pv[c]);
        }
        T qd[9][VO];
        TO q[9][VO];
#pragma unroll
        for (int e = 0; e < VO; ++e) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const cplx<T> zz = z[c * R * N + i0 + e];
                qd[2 * c][e] = zz.x;
                qd[2 * c + 1][e] = zz.y;
            }
            qd[8][e] = z[4 * R * N + i0 + e].x;
#pragma unroll
            for (int c = 0; c < 9; ++c) q[c][e] = (TO)qd[c][e];
        }
        if (MODE == FS_P5_CGF) {
            // r -= alpha q, <r, r> (lanes past the grid update padding only)
#pragma unroll
            for (int c = 0; c < 9; ++c) {
#pragma unroll
                for (int e = 0; e < VO; ++e) pv[c][e] -= alpha * q[c][e];
                stv<VO, TO>(rout + c * cs + v0, pv[c]);
            }
#pragma unroll
            for (int e = 0; e < VO; ++e) {
                if (i0 + e >= nel) continue;
#pragma unroll
                for (int c = 0; c < 9; ++c) acc0 += (T)(pv[c][e] * pv[c][e]);
            }
            continue;
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) stv<VO, TO>(out + c * cs + v0, q[c]);
        if (MODE == FS_P5_PLAIN) continue;
#pragma unroll
        for (int e = 0; e < VO; ++e) {
            if (i0 + e >= nel) continue;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                if (MODE == FS_P5_DOT) {
                    acc0 += (T)(pv[c][e] * q[c][e]);
                } else {
                    acc0 += (T)(q[c][e] * q[c][e]);
                    acc1 += (double)(qd[c][e] * qd[c][e]);
                }
            }
        }
    }
    if (MODE == FS_P5_PLAIN) return;
    const int nb = gridDim.x;
    double part[2];
    part[0] = block_sum((double)acc0);
    if (MODE == FS_P5_CGF) {
        // the block's part of <r, r> (k_cg_rr reduces the parts)
        if (tid == 0) a.partials[blockIdx.x] = part[0];
        return;
    }
    part[1] = (MODE == FS_P5_RHS) ? block_sum(acc1) : 0.0;
    if (!publish_partials<2>(part, a.partials, blockIdx.x, nb, &cg->ticket)) return;
    double tot[2];
    reduce_partials<2>(a.partials, nb, &cg->ticket, tot);
    if (tid != 0) return;
    if (MODE == FS_P5_DOT)
        cg_after_dot(cg, tot[0]);
    else
        cg_start(cg, tot[0], tot[1]);
}

// ------------------------------------------------------------------ launcher
enum FsPassKind : int {
    FK_P1_PLAIN_F64, FK_P1_PLAIN_F32, FK_P1_TAN_F64, FK_P1_TAN_F32, FK_P1_CG_F64, FK_P1_CG_F32,
    FK_P2_F64, FK_P2_F32, FK_P3_F64, FK_P3_F32, FK_P4_F64, FK_P4_F32,
    FK_P5_PLAIN_F64, FK_P5_PLAIN_F32, FK_P5_DOT_F64, FK_P5_DOT_F32,
    FK_P5_RHS_F64_TO_F64, FK_P5_RHS_F64_TO_F32,
    // double-float FFTs (the mixed path's residual)
    FK_P1_PLAIN_DD, FK_P2_DD, FK_P3_DD, FK_P4_DD, FK_P5_RHS_DD_TO_F32, FK_P5_PLAIN_DD_TO_F64,
    // right-hand sides of the macroscopic tangent
    FK_P1_TANRHS_F64, FK_P1_TANRHS_F32, FK_P5_RHS_F32_TO_F32,
    // the CG iteration without the update pass (FS_P1_CGF / FS_P5_CGF), FP32
    FK_P1_CGF_F32, FK_P5_CGF_F32,
    FK_COUNT
};

int fs_row_blocks(int N, bool fp64);

cudaError_t run_fs_pass(int N, FsPassKind kind, const FsArgs& a, cudaStream_t s);

template <int N>
cudaError_t run_fs_pass_n(FsPassKind kind, const FsArgs& a, cudaStream_t s);

template <typename K>
static cudaError_t launch_fs(K kernel, dim3 grid, int threads, size_t smem, const FsArgs& a, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// The x2 passes are the small-strain kernels over nine components; they
// read the spectrum, the twiddles and (when set) the CG state.
template <int N, typename T, bool FWD>
static cudaError_t launch_fs_p24(const FsArgs& a, cudaStream_t s) {
    using C = Cfg<N, T>;
    PassArgs b{};
    b.out = a.out;
    b.cg = a.cg;
    b.tw = a.tw;
    b.red_in = a.red_in;
    b.red_n = a.red_n;
    const dim3 g((C::H + C::W2 - 1) / C::W2, (kFsComp * N + C::S2 - 1) / C::S2, 1);
    cudaError_t e = cudaFuncSetAttribute(k_p24<N, T, FWD, kFsComp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_p24);
    if (e != cudaSuccess) return e;
    k_p24<N, T, FWD, kFsComp><<<g, C::T2, C::smem_p24, s>>>(b);
    return cudaGetLastError();
}

template <int N>
cudaError_t run_fs_pass_n(FsPassKind kind, const FsArgs& a, cudaStream_t s) {
    using C32 = FsCfg<N, float>;
    using C64 = FsCfg<N, double>;
    using CDD = FsCfg<N, dd>;
    static_assert(CDD::row_blocks == C64::row_blocks && CDD::W3 == C64::W3,
                  "double-float passes share the FP64 geometry");
    const dim3 r32(C32::row_blocks), r64(C64::row_blocks);
    const dim3 g32((C32::H + C32::W3 - 1) / C32::W3, N), g64((C64::H + C64::W3 - 1) / C64::W3, N);
    const size_t m32 = C32::smem_rows, m64 = C64::smem_rows;
    switch (kind) {
        case FK_P1_PLAIN_F64: return launch_fs(k_fs_p1<N, double, FS_P1_PLAIN>, r64, kThreads, m64, a, s);
        case FK_P1_PLAIN_F32: return launch_fs(k_fs_p1<N, float, FS_P1_PLAIN>, r32, kThreads, m32, a, s);
        case FK_P1_TAN_F64: return launch_fs(k_fs_p1<N, double, FS_P1_TAN>, r64, kThreads, m64, a, s);
        case FK_P1_TAN_F32: return launch_fs(k_fs_p1<N, float, FS_P1_TAN>, r32, kThreads, m32, a, s);
        case FK_P1_CG_F64: return launch_fs(k_fs_p1<N, double, FS_P1_CG>, r64, kThreads, m64, a, s);
        case FK_P1_CG_F32: return launch_fs(k_fs_p1<N, float, FS_P1_CG>, r32, kThreads, m32, a, s);
        case FK_P2_F64: return launch_fs_p24<N, double, true>(a, s);
        case FK_P2_F32: return launch_fs_p24<N, float, true>(a, s);
        case FK_P4_F64: return launch_fs_p24<N, double, false>(a, s);
        case FK_P4_F32: return launch_fs_p24<N, float, false>(a, s);
        case FK_P3_F64: return launch_fs(k_fs_p3<N, double>, g64, C64::T3, C64::smem_p3, a, s);
        case FK_P3_F32: return launch_fs(k_fs_p3<N, float>, g32, C32::T3, C32::smem_p3, a, s);
        case FK_P5_PLAIN_F64: return launch_fs(k_fs_p5<N, double, FS_P5_PLAIN, double>, r64, kThreads, m64, a, s);
        case FK_P5_PLAIN_F32: return launch_fs(k_fs_p5<N, float, FS_P5_PLAIN, float>, r32, kThreads, m32, a, s);
        case FK_P5_DOT_F64: return launch_fs(k_fs_p5<N, double, FS_P5_DOT, double>, r64, kThreads, m64, a, s);
        case FK_P5_DOT_F32: return launch_fs(k_fs_p5<N, float, FS_P5_DOT, float>, r32, kThreads, m32, a, s);
        case FK_P5_RHS_F64_TO_F64:
            return launch_fs(k_fs_p5<N, double, FS_P5_RHS, double>, r64, kThreads, m64, a, s);
        case FK_P5_RHS_F64_TO_F32:
            return launch_fs(k_fs_p5<N, double, FS_P5_RHS, float>, r64, kThreads, m64, a, s);
        case FK_P1_PLAIN_DD: return launch_fs(k_fs_p1<N, dd, FS_P1_PLAIN>, r64, kThreads, m64, a, s);
        case FK_P2_DD: return launch_fs_p24<N, dd, true>(a, s);
        case FK_P4_DD: return launch_fs_p24<N, dd, false>(a, s);
        case FK_P3_DD: return launch_fs(k_fs_p3<N, dd>, g64, CDD::T3, CDD::smem_p3, a, s);
        case FK_P5_RHS_DD_TO_F32: return launch_fs(k_fs_p5<N, dd, FS_P5_RHS, float>, r64, kThreads, m64, a, s);
        case FK_P5_PLAIN_DD_TO_F64:
            return launch_fs(k_fs_p5<N, dd, FS_P5_PLAIN, double>, r64, kThreads, m64, a, s);
        case FK_P1_TANRHS_F64: return launch_fs(k_fs_p1<N, double, FS_P1_TANRHS>, r64, kThreads, m64, a, s);
        case FK_P1_TANRHS_F32: return launch_fs(k_fs_p1<N, float, FS_P1_TANRHS>, r32, kThreads, m32, a, s);
        case FK_P5_RHS_F32_TO_F32:
            return launch_fs(k_fs_p5<N, float, FS_P5_RHS, float>, r32, kThreads, m32, a, s);
        case FK_P1_CGF_F32: return launch_fs(k_fs_p1<N, float, FS_P1_CGF>, r32, kThreads, m32, a, s);
        case FK_P5_CGF_F32: return launch_fs(k_fs_p5<N, float, FS_P5_CGF, float>, r32, kThreads, m32, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftg
