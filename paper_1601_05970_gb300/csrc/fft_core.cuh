// Odd-radix (3, 5) FFT building blocks for sm_103a.
//
// A pencil of length N = N1 * N2 is transformed in two register stages with
// one shared-memory exchange between them (a Stockham-style four-step
// decomposition; the DFT pair is that of Eq. (DFT_forward_inverse), with the
// 1/|N| factor applied by the caller):
//
//   index n = t + N2*m  (t < N2, m < N1),   frequency k = k1 + N1*k2
//   stage A : for each t, an N1-point DFT over m, then the twiddle w_N^{t k1}
//   stage B : for each k1, an N2-point DFT over t
//
// Stage A leaves Y_t[k1] at position t + N2*k1; stage B reads the N2 values
// at positions N2*k1 + t and writes frequency k1 + N1*k2 either in natural
// order or back in place at position N2*k1 + k2 (the "permuted" order used
// when the spectrum stays in shared memory). Every stage reads and writes
// the same set of positions, so each runs in place without a barrier inside.
// The inverse runs the same stages backwards with conjugate twiddles.
//
// Inside a stage the N1- or N2-point DFT runs in registers, itself split
// recursively into radix-3 and radix-5 butterflies whose twiddles come from
// the same table w_N^j (read with warp-uniform indices, i.e. broadcast).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dd.cuh"

// Twiddles inside the FP32 register DFTs: 1 = compile-time constants
// (immediate operands), 0 = read from the shared-memory table. FP64 DFTs
// always read the table (measured faster at 243^3: 3.14 against 3.19 ms for
// the FP64 x3 pass, while the FP32 passes gain 1-2 % from immediates).
#ifndef FFTG_TWIMM
#define FFTG_TWIMM 1
#endif

namespace fftg {

template <typename T>
struct __align__(2 * sizeof(T)) cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.x, -a.y); }
// i * a
template <typename T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> a) { return mk(-a.y, a.x); }

// Multiply by the table twiddle w = exp(-2 pi i j/N) for the forward
// direction (S = -1) or by its conjugate for the inverse (S = +1).
template <int S, typename T>
__device__ __forceinline__ cplx<T> twmul(cplx<T> v, cplx<T> w) {
    return S < 0 ? cmul(v, w) : cmulc(v, w);
}

// x / 2, and -x where S < 0: exact operations. For double-float pairs both
// words are scaled or negated, which gives the same bits as the general
// double-float product by 0.5 or by +-1 at a fraction of its cost.
template <typename T>
__device__ __forceinline__ cplx<T> half_of(cplx<T> a) { return T(0.5) * a; }
template <>
__device__ __forceinline__ cplx<dd> half_of<dd>(cplx<dd> a) {
    return mk(dd(0.5f * a.x.hi, 0.5f * a.x.lo), dd(0.5f * a.y.hi, 0.5f * a.y.lo));
}
template <int S, typename T>
__device__ __forceinline__ cplx<T> signed_by(cplx<T> a) {
    if constexpr (S < 0) return mk(-a.x, -a.y);
    else return a;
}

// ---------------------------------------------------------------- butterflies
// DFT of 3 or 5 points with kernel exp(S * 2 pi i jk / P), in place.
template <int P, int S, typename T>
struct Butterfly;

template <int S, typename T>
struct Butterfly<3, S, T> {
    static __device__ __forceinline__ void run(cplx<T>* a) {
        const T h = T(0.86602540378443864676);  // sqrt(3)/2
        cplx<T> t1 = a[1] + a[2];
        cplx<T> t2 = a[1] - a[2];
        cplx<T> m = a[0] - half_of(t1);
        cplx<T> r = mul_i(t2);
        r = h * signed_by<S>(r);
        a[0] = a[0] + t1;
        a[1] = m + r;
        a[2] = m - r;
    }
};

template <int S, typename T>
struct Butterfly<5, S, T> {
    static __device__ __forceinline__ void run(cplx<T>* a) {
        const T c1 = T(0.30901699437494742410);   // cos(2 pi/5)
        const T c2 = T(-0.80901699437494742410);  // cos(4 pi/5)
        const T s1 = T(0.95105651629515357212);   // sin(2 pi/5)
        const T s2 = T(0.58778525229247312917);   // sin(4 pi/5)
        cplx<T> b1 = a[1] + a[4], b2 = a[2] + a[3];
        cplx<T> d1 = a[1] - a[4], d2 = a[2] - a[3];
        cplx<T> A1 = a[0] + c1 * b1 + c2 * b2;
        cplx<T> A2 = a[0] + c2 * b1 + c1 * b2;
        cplx<T> B1 = mul_i(s1 * d1 + s2 * d2);
        cplx<T> B2 = mul_i(s2 * d1 - s1 * d2);
        B1 = signed_by<S>(B1);
        B2 = signed_by<S>(B2);
        a[0] = a[0] + b1 + b2;
        a[1] = A1 + B1;
        a[4] = A1 - B1;
        a[2] = A2 + B2;
        a[3] = A2 - B2;
    }
};

// ------------------------------------------------------- constant twiddles
// cos and sin of 2 pi j / n at compile time: the angle is reduced by whole
// quarter turns (exact integer arithmetic) to |phi| <= pi/4, where the
// Taylor series of sin and cos converge to double precision in a few terms,
// and rotated back.
constexpr double cx_sin_series(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 12; ++k) {
        term *= -x * x / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
constexpr double cx_cos_series(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 12; ++k) {
        term *= -x * x / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}
// which = 0: cos(2 pi j / n), 1: sin(2 pi j / n); 0 <= j < n
constexpr double cx_trig2pi(int j, int n, int which) {
    const int q = (8 * j + n) / (2 * n);  // nearest whole quarter turn
    const int r = 4 * j - q * n;          // |r| <= n / 2
    const double phi = 1.5707963267948966192313216916398 * double(r) / double(n);
    const double c = cx_cos_series(phi), s = cx_sin_series(phi);
    switch (q & 3) {
        case 0: return which ? s : c;
        case 1: return which ? c : -s;
        case 2: return which ? -s : -c;
        default: return which ? -c : s;
    }
}

// v * exp(S * 2 pi i J / N) with the factors as immediate constants
template <int N, int J, int S, typename T>
__device__ __forceinline__ cplx<T> twmul_c(cplx<T> v) {
    constexpr T c = T(cx_trig2pi(J, N, 0));
    constexpr T s = T(S * cx_trig2pi(J, N, 1));
    return mk(v.x * c - v.y * s, v.x * s + v.y * c);
}

// f(integral_constant<int, I>) for I = B, ..., E - 1, unrolled at compile time
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------- register DFT
// R-point DFT in registers (R = 3^a 5^b), natural order in and out.
// Split R = P*Q with P the smallest factor: n = q + Q*p, k = k1 + P*k2.
template <int N, int R, int S, typename T>
struct RegDFT {
    static __device__ __forceinline__ void run(cplx<T> (&a)[R], const cplx<T>* __restrict__ tw) {
        constexpr int P = (R % 3 == 0) ? 3 : 5;
        constexpr int Q = R / P;
        static_assert(P * Q == R, "R must be a product of 3 and 5");
        cplx<T> y[R];
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            cplx<T> v[P];
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = a[q + Q * p];
            Butterfly<P, S, T>::run(v);
            static_for<0, P>([&](auto kc) {
                constexpr int k1 = decltype(kc)::value;
                constexpr int j = (q * k1 * (N / R)) % N;  // 0 iff q * k1 == 0
                if constexpr (j == 0) {
                    y[k1 * Q + q] = v[k1];
                } else if constexpr (FFTG_TWIMM && sizeof(T) == 4) {
                    y[k1 * Q + q] = twmul_c<N, j, S, T>(v[k1]);
                } else {
                    y[k1 * Q + q] = twmul<S>(v[k1], tw[j]);
                }
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            cplx<T> z[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) z[q] = y[k1 * Q + q];
            RegDFT<N, Q, S, T>::run(z, tw);
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) a[k1 + P * k2] = z[k2];
        }
    }
};

template <int N, int S, typename T>
struct RegDFT<N, 1, S, T> {
    static __device__ __forceinline__ void run(cplx<T> (&)[1], const cplx<T>* __restrict__) {}
};

// ---------------------------------------------------------------- plans
// N = N1 * N2: N1 points per thread in stage A, N2 in stage B.
template <int N>
struct Plan;
#define FFTG_PLAN(n, a, b)                          \
    template <>                                     \
    struct Plan<n> {                                \
        static constexpr int N1 = a, N2 = b;        \
    };
FFTG_PLAN(3, 3, 1)
FFTG_PLAN(5, 5, 1)
FFTG_PLAN(9, 9, 1)
FFTG_PLAN(15, 15, 1)
FFTG_PLAN(25, 25, 1)
FFTG_PLAN(27, 27, 1)
FFTG_PLAN(45, 9, 5)
FFTG_PLAN(75, 15, 5)
FFTG_PLAN(81, 9, 9)
FFTG_PLAN(125, 25, 5)
FFTG_PLAN(135, 15, 9)
FFTG_PLAN(225, 15, 15)
FFTG_PLAN(243, 27, 9)
#undef FFTG_PLAN

// Radix schedules other than the default split N = N1 * N2 (the kernels
// take N1 as a template parameter; N2 = N / N1). A schedule is valid when
// N1 divides N and both factors are products of 3 and 5.
constexpr bool radix35(int n) {
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    return n == 1;
}
constexpr bool valid_split(int N, int N1) { return N1 >= 1 && N % N1 == 0 && radix35(N1) && radix35(N / N1); }

// position of frequency k after a forward stage B in permuted mode
template <int N, int N1 = Plan<N>::N1>
__device__ __forceinline__ int perm_pos(int k) {
    constexpr int N2 = N / N1;
    return N2 * (k % N1) + k / N1;
}

// ---------------------------------------------------------------- stages
// src/dst: pencil base pointers; ss/ds: element strides (in cplx units).
// Each stage exists for the default split (Plan<N>) and, with the first
// factor N1 given explicitly, for any valid split.

// forward stage A: reads positions t + N2*m, writes t + N2*k1 (with twiddle)
template <int N, int N1, typename T>
__device__ __forceinline__ void fwdA(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int t,
                                     const cplx<T>* __restrict__ tw) {
    static_assert(valid_split(N, N1), "radix schedule");
    constexpr int N2 = N / N1;
    cplx<T> v[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) v[m] = src[(t + N2 * m) * ss];
    RegDFT<N, N1, -1, T>::run(v, tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        cplx<T> y = v[k1];
        if (N2 > 1 && k1 > 0) y = twmul<-1>(y, tw[t * k1]);  // t*k1 < N1*N2 = N
        dst[(t + N2 * k1) * ds] = y;
    }
}

// forward stage B: reads N2*k1 + q; NATURAL: writes k1 + N1*k2, else N2*k1 + k2
template <int N, int N1, bool NATURAL, typename T>
__device__ __forceinline__ void fwdB(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int k1,
                                     const cplx<T>* __restrict__ tw) {
    constexpr int N2 = N / N1;
    cplx<T> v[N2];
#pragma unroll
    for (int q = 0; q < N2; ++q) v[q] = src[(N2 * k1 + q) * ss];
    RegDFT<N, N2, -1, T>::run(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) dst[(NATURAL ? (k1 + N1 * k2) : (N2 * k1 + k2)) * ds] = v[k2];
}

// inverse stage B': NATURAL: reads k1 + N1*k2, else N2*k1 + k2;
// writes N2*k1 + t with the conjugate twiddle
template <int N, int N1, bool NATURAL, typename T>
__device__ __forceinline__ void invB(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int k1,
                                     const cplx<T>* __restrict__ tw) {
    constexpr int N2 = N / N1;
    cplx<T> v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = src[(NATURAL ? (k1 + N1 * k2) : (N2 * k1 + k2)) * ss];
    RegDFT<N, N2, +1, T>::run(v, tw);
#pragma unroll
    for (int t = 0; t < N2; ++t) {
        cplx<T> z = v[t];
        if (k1 > 0 && t > 0) z = twmul<+1>(z, tw[t * k1]);  // t*k1 < N
        dst[(N2 * k1 + t) * ds] = z;
    }
}

// inverse stage A': reads t + N2*k1, writes t + N2*m
template <int N, int N1, typename T>
__device__ __forceinline__ void invA(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int t,
                                     const cplx<T>* __restrict__ tw) {
    constexpr int N2 = N / N1;
    cplx<T> v[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[(t + N2 * k1) * ss];
    RegDFT<N, N1, +1, T>::run(v, tw);
#pragma unroll
    for (int m = 0; m < N1; ++m) dst[(t + N2 * m) * ds] = v[m];
}

// the stages with the default split
template <int N, typename T>
__device__ __forceinline__ void fwdA(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int t,
                                     const cplx<T>* __restrict__ tw) {
    fwdA<N, Plan<N>::N1, T>(src, ss, dst, ds, t, tw);
}
template <int N, bool NATURAL, typename T>
__device__ __forceinline__ void fwdB(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int k1,
                                     const cplx<T>* __restrict__ tw) {
    fwdB<N, Plan<N>::N1, NATURAL, T>(src, ss, dst, ds, k1, tw);
}
template <int N, bool NATURAL, typename T>
__device__ __forceinline__ void invB(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int k1,
                                     const cplx<T>* __restrict__ tw) {
    invB<N, Plan<N>::N1, NATURAL, T>(src, ss, dst, ds, k1, tw);
}
template <int N, typename T>
__device__ __forceinline__ void invA(const cplx<T>* src, int ss, cplx<T>* dst, int ds, int t,
                                     const cplx<T>* __restrict__ tw) {
    invA<N, Plan<N>::N1, T>(src, ss, dst, ds, t, tw);
}

}  // namespace fftg
