// Double-float numbers: the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, about 48 significant bits (relative rounding
// near 2^-47, some 7e-15).
//
// The arithmetic is built from the error-free transformations of Dekker
// ("A floating-point technique for extending the available precision",
// 1971) and Knuth (TAOCP vol. 2, 4.2.2):
//   TwoSum(a, b)     = (s, e) with s = fl(a + b) and a + b = s + e exactly;
//   FastTwoSum(a, b) = the same in three operations when |a| >= |b|;
//   TwoProd(a, b)    = (p, e) with p = fl(a b) and a b = p + e exactly,
//                      e = fma(a, b, -p).
// Addition is Dekker's: TwoSum of the high parts, the low parts added to
// the error term, renormalised by FastTwoSum; its error is a few units of
// 2^-47 of |a| + |b|, which suits an FFT (whose rounding error scales with
// the norm of its input anyway). Multiplication is TwoProd plus the cross
// terms.
//
// The residual pass of the mixed-precision path runs its FFTs in this
// format: GB300 executes FP32 at many times its FP64 rate, and the residual
// only needs accuracy well below the CG roundoff floor (1e-13 of ||sigma||).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace fftg {

struct __align__(8) dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to v: hi = fl32(v), lo = fl32(v - hi)
    __host__ __device__ constexpr dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ constexpr explicit dd(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ constexpr explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ constexpr explicit operator float() const { return hi + lo; }
};

// Round-to-nearest FP32 primitives that the compiler may not fuse or
// reorder: the CUDA intrinsics on the device, plain IEEE float arithmetic
// (and std::fma) on the host, where the arithmetic is tested.
__host__ __device__ __forceinline__ float dd_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float s = a + b;
    return s;
#endif
}
__host__ __device__ __forceinline__ float dd_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float s = a - b;
    return s;
#endif
}
__host__ __device__ __forceinline__ float dd_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float s = a * b;
    return s;
#endif
}
__host__ __device__ __forceinline__ float dd_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

// TwoSum: s + e = a + b exactly
__host__ __device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = dd_add(a, b);
    const float bb = dd_sub(s, a);
    const float e = dd_add(dd_sub(a, dd_sub(s, bb)), dd_sub(b, bb));
    return dd(s, e);
}

// FastTwoSum: s + e = a + b exactly when |a| >= |b|
__host__ __device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
    const float s = dd_add(a, b);
    return dd(s, dd_sub(b, dd_sub(s, a)));
}

// TwoProd: p + e = a b exactly
__host__ __device__ __forceinline__ dd dd_two_prod(float a, float b) {
    const float p = dd_mul(a, b);
    return dd(p, dd_fma(a, b, -p));
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
    const dd s = dd_two_sum(a.hi, b.hi);
    return dd_fast_two_sum(s.hi, dd_add(s.lo, dd_add(a.lo, b.lo)));
}

__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }

__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
    const dd p = dd_two_prod(a.hi, b.hi);
    float e = dd_fma(a.hi, b.lo, p.lo);
    e = dd_fma(a.lo, b.hi, e);
    return dd_fast_two_sum(p.hi, e);
}

__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }

__host__ __device__ __forceinline__ bool operator>(dd a, dd b) {
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__host__ __device__ __forceinline__ bool operator<(dd a, dd b) { return b > a; }

#ifdef __CUDACC__
// 1/sqrt(x) for the per-frequency factors of Ghat (FP64 rsqrt, rounded)
__device__ __forceinline__ dd rsqrt_t(dd x) { return dd(rsqrt((double)x)); }
#endif

}  // namespace fftg
