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
#include "fft_core.cuh"

namespace fftg {

enum : int { P1_PLAIN = 0, P1_TAN = 1, P1_CG = 2, P1_TANRHS = 3 };
enum : int { P5_PLAIN = 0, P5_DOT = 1, P5_RHS = 2 };

struct PassArgs {
    const void* in;        // P1: real field; P2-P4: unused; P5: spectrum
    void* out;             // P1: spectrum; P2-P4: spectrum (in place); P5: real field
    const void* aux;       // P1_CG: r; P5_DOT: p
    void* aux2;            // P1_CG: p (updated in place)
    const void* tangent;   // [7][V]: K, 2G_eff, w11, w22, w23, w13, w12
    CGState* cg;           // per field, or null
    double* partials;      // [nf][nblocks][2]
    const void* tw;        // w_N^j, j < N, in the FFT precision
    double scale;          // P3: factor on Ghat (+-1/N^3)
    long long fstride;     // real-field stride between fields (elements)
    long long sstride;     // spectrum stride between fields (complex elements)
    long long tstride;     // tangent stride between fields (0: shared)
};

template <int N, typename T>
struct Cfg {
    static constexpr int H = (N + 1) / 2;
    static constexpr int CS = (int)sizeof(cplx<T>);
    static constexpr int BUDGET = 100 * 1024;
    static constexpr int fl2(int x) {
        return x >= 64 ? 64 : x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1;
    }
    static constexpr int R = fl2(BUDGET / (3 * N * CS));                      // rows, P1/P5
    static constexpr int W3 = fl2(BUDGET / (6 * N * CS)) > 32 ? 32 : fl2(BUDGET / (6 * N * CS));
    static constexpr int W2 = (CS == 8) ? 32 : 16;                            // columns, P2/P4
    static constexpr int S2 = fl2(BUDGET / (N * W2 * CS)) > 16 ? 16 : fl2(BUDGET / (N * W2 * CS));
    static constexpr size_t smem_rows = (size_t)(3 * R * N + N) * CS;
    static constexpr size_t smem_p3 = (size_t)(6 * W3 * N + N) * CS;
    static constexpr size_t smem_p24 = (size_t)(S2 * W2 * N + N) * CS;
    static constexpr int row_blocks = (N * N + R - 1) / R;
};

template <typename T>
__device__ __forceinline__ void load_tw(cplx<T>* tw, const void* src, int n) {
    const cplx<T>* s = (const cplx<T>*)src;
    for (int i = threadIdx.x; i < n; i += kThreads) tw[i] = s[i];
}

// s = C : p with the compact J2 tangent (Section 4.2):
// C = K I(x)I + 2G_eff I_d - w (x) w,  w = sqrt(-b) N, b < 0
template <typename T>
__device__ __forceinline__ void apply_tangent(const T* __restrict__ tg, long long v, long long V,
                                              const T (&p)[6], T (&s)[6]) {
    const T K = tg[v], g2 = tg[V + v];
    const T w0 = tg[2 * V + v], w1 = tg[3 * V + v], w3 = tg[4 * V + v], w4 = tg[5 * V + v],
            w5 = tg[6 * V + v];
    const T w2 = -(w0 + w1);
    const T tr = p[0] + p[1] + p[2];
    const T m = tr * T(1.0 / 3.0);
    const T wp = w0 * p[0] + w1 * p[1] + w2 * p[2] + T(2) * (w3 * p[3] + w4 * p[4] + w5 * p[5]);
    const T kt = K * tr;
    s[0] = kt + g2 * (p[0] - m) - wp * w0;
    s[1] = kt + g2 * (p[1] - m) - wp * w1;
    s[2] = kt + g2 * (p[2] - m) - wp * w2;
    s[3] = g2 * p[3] - wp * w3;
    s[4] = g2 * p[4] - wp * w4;
    s[5] = g2 * p[5] - wp * w5;
}

// ----------------------------------------------------------------------- P1
template <int N, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_p1(PassArgs a) {
    using C = Cfg<N, T>;
    constexpr int R = C::R, H = C::H;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [3][R][N]
    const int f = blockIdx.z;
    if (MODE == P1_CG && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const long long V = (long long)N * N * N;
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const T* in = (const T*)a.in + f * a.fstride;
    const T* tg = (const T*)a.tangent + f * a.tstride;
    T beta = T(0);
    bool first = true;  // first CG iteration: p = r (p holds no data yet)
    if (MODE == P1_CG) {
        beta = (T)a.cg[f].beta;
        first = a.cg[f].it == 0;
    }
    for (int i = tid; i < R * N; i += kThreads) {
        T s[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (i < nel) {
            const long long v = base + i;
            T p[6];
            if (MODE == P1_CG) {
                const T* r = (const T*)a.aux + f * a.fstride;
                T* pp = (T*)a.aux2 + f * a.fstride;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const T pv = first ? r[c * V + v] : r[c * V + v] + beta * pp[c * V + v];
                    pp[c * V + v] = pv;
                    p[c] = pv;
                }
            } else if (MODE == P1_TANRHS) {
#pragma unroll
                for (int c = 0; c < 6; ++c) p[c] = (c == f) ? T(1) : T(0);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) p[c] = in[c * V + v];
            }
            if (MODE == P1_PLAIN) {
#pragma unroll
                for (int c = 0; c < 6; ++c) s[c] = p[c];
            } else {
                apply_tangent<T>(tg, v, V, p, s);
            }
        }
        z[i] = mk(s[0], s[1]);
        z[R * N + i] = mk(s[2], s[3]);
        z[2 * R * N + i] = mk(s[4], s[5]);
    }
    __syncthreads();
    constexpr int NP = 3 * R;
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
    cplx<T>* out = (cplx<T>*)a.out + f * a.sstride;
    const long long HS = (long long)N * N * H;
    for (int it = tid; it < nrows * H; it += kThreads) {
        const int row = it / H, k = it - row * H;
        const int pk = perm_pos<N>(k), pn = perm_pos<N>(k == 0 ? 0 : N - k);
        const long long o = (long long)(row0 + row) * H + k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<T> zk = z[(c * R + row) * N + pk];
            const cplx<T> zn = conj(z[(c * R + row) * N + pn]);
            const cplx<T> A = T(0.5) * (zk + zn);
            const cplx<T> d = zk - zn;  // (zk - zn) / (2i) = (d.y, -d.x) / 2
            const cplx<T> B = mk(T(0.5) * d.y, T(-0.5) * d.x);
            out[(2 * c) * HS + o] = A;
            out[(2 * c + 1) * HS + o] = B;
        }
    }
}

// -------------------------------------------------------------- P2 / P4 (x2)
template <int N, typename T, bool FWD>
__global__ void __launch_bounds__(kThreads) k_p24(PassArgs a) {
    using C = Cfg<N, T>;
    constexpr int H = C::H, W = C::W2, S = C::S2;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [S][N][W]
    const int f = blockIdx.z;
    if (a.cg && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, slab0 = blockIdx.y * S;
    cplx<T>* sp = (cplx<T>*)a.out + f * a.sstride;
    constexpr int P = S * W;
    if (FWD) {
        for (int it = tid; it < P * N2; it += kThreads) {
            const int pc = it % P, t = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < 6 * N)
                fwdA<N, T>(sp + (long long)slab * N * H + col, H, buf + s * N * W + w, W, t, tw);
        }
        __syncthreads();
        for (int it = tid; it < P * N1; it += kThreads) {
            const int pc = it % P, k1 = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < 6 * N)
                fwdB<N, true, T>(buf + s * N * W + w, W, sp + (long long)slab * N * H + col, H, k1, tw);
        }
    } else {
        for (int it = tid; it < P * N1; it += kThreads) {
            const int pc = it % P, k1 = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < 6 * N)
                invB<N, true, T>(sp + (long long)slab * N * H + col, H, buf + s * N * W + w, W, k1, tw);
        }
        __syncthreads();
        for (int it = tid; it < P * N2; it += kThreads) {
            const int pc = it % P, t = it / P;
            const int s = pc / W, w = pc - s * W, col = col0 + w, slab = slab0 + s;
            if (col < H && slab < 6 * N)
                invA<N, T>(buf + s * N * W + w, W, sp + (long long)slab * N * H + col, H, t, tw);
        }
    }
}

// Ghat : tau at frequency (f1, f2, f3), times `scale`, for the 6 complex
// components (11, 22, 33, 23, 13, 12) held at stride `cs` in shared memory.
template <typename T>
__device__ __forceinline__ void apply_ghat(cplx<T>* b, int cs, int f1, int f2, int f3, T scale) {
    const T q2 = T(f1) * T(f1) + T(f2) * T(f2) + T(f3) * T(f3);
    if (q2 == T(0)) {
#pragma unroll
        for (int c = 0; c < 6; ++c) b[c * cs] = mk(T(0), T(0));
        return;
    }
    const T inv = T(1) / sqrt(q2);
    const T n0 = T(f1) * inv, n1 = T(f2) * inv, n2 = T(f3) * inv;
    cplx<T> t[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = b[c * cs];
    // v = tau n
    const cplx<T> v0 = n0 * t[0] + n1 * t[5] + n2 * t[4];
    const cplx<T> v1 = n0 * t[5] + n1 * t[1] + n2 * t[3];
    const cplx<T> v2 = n0 * t[4] + n1 * t[3] + n2 * t[2];
    const cplx<T> sn = n0 * v0 + n1 * v1 + n2 * v2;
    b[0 * cs] = scale * (T(2) * n0 * v0 - (n0 * n0) * sn);
    b[1 * cs] = scale * (T(2) * n1 * v1 - (n1 * n1) * sn);
    b[2 * cs] = scale * (T(2) * n2 * v2 - (n2 * n2) * sn);
    b[3 * cs] = scale * (n1 * v2 + n2 * v1 - (n1 * n2) * sn);
    b[4 * cs] = scale * (n0 * v2 + n2 * v0 - (n0 * n2) * sn);
    b[5 * cs] = scale * (n0 * v1 + n1 * v0 - (n0 * n1) * sn);
}

// ------------------------------------------------------------- P3 (x1 + Ghat)
template <int N, typename T>
__global__ void __launch_bounds__(kThreads) k_p3(PassArgs a) {
    using C = Cfg<N, T>;
    constexpr int H = C::H, W = C::W3;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* buf = tw + N;  // [6][N][W]
    const int f = blockIdx.z;
    if (a.cg && a.cg[f].done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    __syncthreads();
    const int col0 = blockIdx.x * W, k2 = blockIdx.y;
    cplx<T>* sp = (cplx<T>*)a.out + f * a.sstride;
    constexpr int P = 6 * W;
    const long long NH = (long long)N * H;
    for (int it = tid; it < P * N2; it += kThreads) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) fwdA<N, T>(sp + c * N * NH + k2 * H + col, (int)NH, buf + c * N * W + w, W, t, tw);
    }
    __syncthreads();
    if (N2 > 1) {
        for (int it = tid; it < P * N1; it += kThreads) {
            const int pc = it % P, k1 = it / P;
            const int c = pc / W, w = pc - c * W;
            if (col0 + w < H) fwdB<N, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
        }
        __syncthreads();
    }
    const int f2 = (k2 <= (N - 1) / 2) ? k2 : k2 - N;
    for (int it = tid; it < N * W; it += kThreads) {
        const int pos = it / W, w = it - pos * W, col = col0 + w;
        if (col < H) {
            const int kk = (pos / N2) + N1 * (pos % N2);
            const int f1 = (kk <= (N - 1) / 2) ? kk : kk - N;
            apply_ghat<T>(buf + pos * W + w, N * W, f1, f2, col, (T)a.scale);
        }
    }
    __syncthreads();
    if (N2 > 1) {
        for (int it = tid; it < P * N1; it += kThreads) {
            const int pc = it % P, k1 = it / P;
            const int c = pc / W, w = pc - c * W;
            if (col0 + w < H) invB<N, false, T>(buf + c * N * W + w, W, buf + c * N * W + w, W, k1, tw);
        }
        __syncthreads();
    }
    for (int it = tid; it < P * N2; it += kThreads) {
        const int pc = it % P, t = it / P;
        const int c = pc / W, w = pc - c * W, col = col0 + w;
        if (col < H) invA<N, T>(buf + c * N * W + w, W, sp + c * N * NH + k2 * H + col, (int)NH, t, tw);
    }
}

// ----------------------------------------------------------------------- P5
// T: FFT precision; TO: output real type (P5_RHS writes the CG residual r
// in the inner precision).
template <int N, typename T, int MODE, typename TO>
__global__ void __launch_bounds__(kThreads) k_p5(PassArgs a) {
    using C = Cfg<N, T>;
    constexpr int R = C::R, H = C::H;
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* tw = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* z = tw + N;  // [3][R][N]
    const int f = blockIdx.z;
    CGState* cg = a.cg ? a.cg + f : nullptr;
    if (MODE == P5_DOT && cg->done) return;
    const int tid = threadIdx.x;
    load_tw<T>(tw, a.tw, N);
    const long long V = (long long)N * N * N;
    const int row0 = blockIdx.x * R;
    const int nrows = min(R, N * N - row0);
    const long long base = (long long)row0 * N;
    const int nel = nrows * N;
    const cplx<T>* in = (const cplx<T>*)a.in + f * a.sstride;
    const long long HS = (long long)N * N * H;
    for (int it = tid; it < nrows * H; it += kThreads) {
        const int row = it / H, k = it - row * H;
        const long long o = (long long)(row0 + row) * H + k;
        const int pk = perm_pos<N>(k);
        const int pn = perm_pos<N>(k == 0 ? 0 : N - k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<T> A = in[(2 * c) * HS + o], B = in[(2 * c + 1) * HS + o];
            z[(c * R + row) * N + pk] = mk(A.x - B.y, A.y + B.x);  // A + iB
            if (k > 0) z[(c * R + row) * N + pn] = mk(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
        }
    }
    __syncthreads();
    constexpr int NP = 3 * R;
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
    TO* out = (TO*)a.out + f * a.fstride;
    T acc0 = T(0);
    double acc1 = 0.0;
    for (int i = tid; i < nel; i += kThreads) {
        const long long v = base + i;
        const cplx<T> z0 = z[i], z1 = z[R * N + i], z2 = z[2 * R * N + i];
        const T q[6] = {z0.x, z0.y, z1.x, z1.y, z2.x, z2.y};
        if (MODE == P5_DOT) {
            const T* p = (const T*)a.aux + f * a.fstride;
            T pv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                out[c * V + v] = (TO)q[c];
                pv[c] = p[c * V + v];
            }
            acc0 += frob<T>(pv, q);
        } else if (MODE == P5_RHS) {
            TO r[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                r[c] = (TO)q[c];
                out[c * V + v] = r[c];
            }
            acc1 += (double)frob<T>(q, q);
            acc0 += (T)frob<TO>(r, r);
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) out[c * V + v] = (TO)q[c];
        }
    }
    if (MODE == P5_PLAIN) return;
    const int nb = gridDim.x;
    double part[2];
    part[0] = block_sum((double)acc0);
    part[1] = (MODE == P5_RHS) ? block_sum(acc1) : 0.0;
    double* partials = a.partials + (size_t)f * nb * 2;
    if (!publish_partials<2>(part, partials, blockIdx.x, nb, &cg->ticket)) return;
    double tot[2];
    reduce_partials<2>(partials, nb, &cg->ticket, tot);
    if (tid != 0) return;
    if (MODE == P5_DOT) {
        const double pq = tot[0];
        cg->pq = pq;
        if (!isfinite(pq)) {
            cg->done = CG_BREAKDOWN;
        } else if (!(pq > 0.0)) {
            cg->done = cg->stag_window > 0 ? CG_STAGNATED : CG_BREAKDOWN;
        } else {
            cg->alpha = cg->rr / pq;
        }
    } else {
        const double rr = tot[0], gs2 = tot[1];
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
}

// ------------------------------------------------------------------ launcher
enum PassKind : int {
    PK_P1_PLAIN_F64, PK_P1_PLAIN_F32, PK_P1_TAN_F64, PK_P1_TAN_F32, PK_P1_CG_F64, PK_P1_CG_F32,
    PK_P1_TANRHS_F64, PK_P1_TANRHS_F32,
    PK_P2_F64, PK_P2_F32, PK_P4_F64, PK_P4_F32, PK_P3_F64, PK_P3_F32,
    PK_P5_PLAIN_F64, PK_P5_PLAIN_F32, PK_P5_DOT_F64, PK_P5_DOT_F32,
    PK_P5_RHS_F64_TO_F64, PK_P5_RHS_F64_TO_F32, PK_P5_RHS_F32_TO_F32,
    PK_COUNT
};

// Grid geometry of the row passes (blocks per field): needed by the host to
// size the partial-sum buffer.
int row_blocks(int N, bool fp64);

cudaError_t run_pass(int N, PassKind kind, const PassArgs& a, int nf, cudaStream_t s);

template <int N>
cudaError_t run_pass_n(PassKind kind, const PassArgs& a, int nf, cudaStream_t s);

template <typename K>
static cudaError_t launch_k(K kernel, dim3 grid, size_t smem, const PassArgs& a, cudaStream_t s) {
    static_assert(sizeof(PassArgs) < 4096, "kernel params");
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t run_pass_n(PassKind kind, const PassArgs& a, int nf, cudaStream_t s) {
    using C32 = Cfg<N, float>;
    using C64 = Cfg<N, double>;
    const dim3 r32(C32::row_blocks, 1, nf), r64(C64::row_blocks, 1, nf);
    const dim3 c32((C32::H + C32::W2 - 1) / C32::W2, (6 * N + C32::S2 - 1) / C32::S2, nf);
    const dim3 c64((C64::H + C64::W2 - 1) / C64::W2, (6 * N + C64::S2 - 1) / C64::S2, nf);
    const dim3 g32((C32::H + C32::W3 - 1) / C32::W3, N, nf);
    const dim3 g64((C64::H + C64::W3 - 1) / C64::W3, N, nf);
    switch (kind) {
        case PK_P1_PLAIN_F64: return launch_k(k_p1<N, double, P1_PLAIN>, r64, C64::smem_rows, a, s);
        case PK_P1_PLAIN_F32: return launch_k(k_p1<N, float, P1_PLAIN>, r32, C32::smem_rows, a, s);
        case PK_P1_TAN_F64: return launch_k(k_p1<N, double, P1_TAN>, r64, C64::smem_rows, a, s);
        case PK_P1_TAN_F32: return launch_k(k_p1<N, float, P1_TAN>, r32, C32::smem_rows, a, s);
        case PK_P1_CG_F64: return launch_k(k_p1<N, double, P1_CG>, r64, C64::smem_rows, a, s);
        case PK_P1_CG_F32: return launch_k(k_p1<N, float, P1_CG>, r32, C32::smem_rows, a, s);
        case PK_P1_TANRHS_F64: return launch_k(k_p1<N, double, P1_TANRHS>, r64, C64::smem_rows, a, s);
        case PK_P1_TANRHS_F32: return launch_k(k_p1<N, float, P1_TANRHS>, r32, C32::smem_rows, a, s);
        case PK_P2_F64: return launch_k(k_p24<N, double, true>, c64, C64::smem_p24, a, s);
        case PK_P2_F32: return launch_k(k_p24<N, float, true>, c32, C32::smem_p24, a, s);
        case PK_P4_F64: return launch_k(k_p24<N, double, false>, c64, C64::smem_p24, a, s);
        case PK_P4_F32: return launch_k(k_p24<N, float, false>, c32, C32::smem_p24, a, s);
        case PK_P3_F64: return launch_k(k_p3<N, double>, g64, C64::smem_p3, a, s);
        case PK_P3_F32: return launch_k(k_p3<N, float>, g32, C32::smem_p3, a, s);
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
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftg
