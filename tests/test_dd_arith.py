"""Host-side pins of the double-float arithmetic (csrc/dd.cuh) used by the
mixed path's residual FFTs: the error-free transformations are exact, and
addition and multiplication are accurate to the format (about 2^-47).

The same source is compiled for the host by nvcc (no GPU needed) and run on
random operands over a wide exponent range; exact references are formed in
long double (64 or more significand bits, enough for sums and products of
two FP32 numbers whose exponents differ by less than 40).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1601_05970_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include "dd.cuh"
using fftg::dd;
typedef long double L;
static L val(dd a) { return (L)a.hi + (L)a.lo; }
int main() {
    std::mt19937_64 g(12345);
    std::uniform_real_distribution<double> m(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-12, 12);
    long long bad_two_sum = 0, bad_two_prod = 0, bad_fast = 0, bad_norm = 0;
    double worst_add = 0, worst_mul = 0, worst_split = 0;
    const int n = 200000;
    for (int i = 0; i < n; ++i) {
        const double x = std::ldexp(m(g), ex(g)), y = std::ldexp(m(g), ex(g));
        const float a = (float)x, b = (float)y;
        dd s = fftg::dd_two_sum(a, b);
        if ((L)s.hi + (L)s.lo != (L)a + (L)b) ++bad_two_sum;
        dd p = fftg::dd_two_prod(a, b);
        if ((L)p.hi + (L)p.lo != (L)a * (L)b) ++bad_two_prod;
        const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = big == a ? b : a;
        dd f = fftg::dd_fast_two_sum(big, small);
        if ((L)f.hi + (L)f.lo != (L)big + (L)small) ++bad_fast;
        const dd A(x), B(y);
        worst_split = std::fmax(worst_split, (double)(std::fabs(val(A) - (L)x) / std::fabs((L)x)));
        const dd S = A + B, P = A * B;
        if (std::fabs(S.lo) > std::ldexp(std::fabs(S.hi), -23)) ++bad_norm;
        const L es = std::fabs(val(S) - (val(A) + val(B))) / (std::fabs(val(A)) + std::fabs(val(B)));
        const L ep = std::fabs(val(P) - val(A) * val(B)) / std::fabs(val(A) * val(B));
        worst_add = std::fmax(worst_add, (double)es);
        worst_mul = std::fmax(worst_mul, (double)ep);
    }
    std::printf("%lld %lld %lld %lld %.3e %.3e %.3e\n", bad_two_sum, bad_two_prod, bad_fast, bad_norm,
                worst_split, worst_add, worst_mul);
    return 0;
}
"""


def test_double_float_arithmetic(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "dd_host.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "dd_host"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                    "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    bad_two_sum, bad_two_prod, bad_fast, bad_norm = map(int, out[:4])
    worst_split, worst_add, worst_mul = map(float, out[4:])
    assert bad_two_sum == 0 and bad_two_prod == 0 and bad_fast == 0   # error-free: exact
    assert bad_norm == 0                                              # |lo| <= ulp(hi)
    assert worst_split <= 2.0 ** -47                                  # nearest double-float
    assert worst_add <= 2.0 ** -44                                    # Dekker addition
    assert worst_mul <= 2.0 ** -44                                    # product with cross terms
    # and not merely FP32 (2^-24)
    assert max(worst_add, worst_mul) > 0.0


EXACT = r"""
#include <cstdio>
#include <cmath>
#include <cstring>
#include <random>
#include "dd.cuh"
using fftg::dd;
static bool same(dd a, dd b) { return std::memcmp(&a, &b, sizeof(dd)) == 0; }
int main() {
    std::mt19937_64 g(4242);
    std::uniform_real_distribution<double> m(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-30, 30);
    long long bad_half = 0, bad_neg = 0, bad_twice = 0;
    const dd half(0.5), minus1(-1), two(2);
    for (int i = 0; i < 200000; ++i) {
        const dd x(std::ldexp(m(g), ex(g)));
        if (!same(half * x, dd(0.5f * x.hi, 0.5f * x.lo))) ++bad_half;
        if (!same(minus1 * x, -x)) ++bad_neg;
        if (!same(two * x, x + x)) ++bad_twice;
    }
    std::printf("%lld %lld %lld\n", bad_half, bad_neg, bad_twice);
    return 0;
}
"""


def test_exact_scalings_match_the_general_products(tmp_path):
    """The butterflies, the real-to-complex split and Ghat halve, negate and
    double double-float pairs word by word instead of multiplying by 0.5,
    -1 and 2: on normalised pairs the general product gives the same bits."""
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "exact_host.cu"
    src.write_text(EXACT)
    exe = tmp_path / "exact_host"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
                    "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert list(map(int, out)) == [0, 0, 0]
