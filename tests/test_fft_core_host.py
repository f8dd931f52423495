"""The pencil-FFT building blocks of csrc/fft_core.cuh on the host, for every
compiled plan (N = N1 * N2) in FP64 and FP32, against numpy's FFT.

The header is compiled unchanged by the host C++ compiler, with a stub for
the CUDA qualifiers; the stages are chained as the pass kernels chain them:
stage A for every t, then stage B in natural order (forward), and the
inverse stages back (the unnormalised inverse returns N times the input).
The permuted order of stage B (kept in shared memory by P1, P3 and P5) is
checked through perm_pos and a permuted round trip. No GPU is needed.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1601_05970_gb300", "csrc")
GRIDS = (3, 5, 9, 15, 25, 27, 45, 75, 81, 125, 135, 225, 243)

STUB = """#pragma once
#define __device__
#define __host__
#define __forceinline__ inline
#define __align__(n) alignas(n)
"""

HARNESS = r"""
#include <cstdio>
#include <cmath>
#include <vector>
#include "fft_core.cuh"
#include "host_common.h"
using namespace fftg;

template <int N, typename T>
void run(FILE* f) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    std::vector<double> t64(2 * N);
    std::vector<float> t32(2 * N);
    twiddles(N, t64.data(), t32.data());
    std::vector<cplx<T>> tw(N), x(N), a(N), y(N), b(N), z(N), p(N);
    for (int j = 0; j < N; ++j) {
        tw[j].x = sizeof(T) == 8 ? (T)t64[2 * j] : (T)t32[2 * j];
        tw[j].y = sizeof(T) == 8 ? (T)t64[2 * j + 1] : (T)t32[2 * j + 1];
        x[j].x = (T)std::sin(0.7 * j + 0.3 * N);   // deterministic input
        x[j].y = (T)std::cos(1.3 * j * j / (double)N);
    }
    // forward: stage A for every t, then stage B in natural order
    for (int t = 0; t < N2; ++t) fwdA<N, T>(x.data(), 1, a.data(), 1, t, tw.data());
    for (int k1 = 0; k1 < N1; ++k1) fwdB<N, true, T>(a.data(), 1, y.data(), 1, k1, tw.data());
    // inverse from natural order: stage B', then stage A'
    for (int k1 = 0; k1 < N1; ++k1) invB<N, true, T>(y.data(), 1, b.data(), 1, k1, tw.data());
    for (int t = 0; t < N2; ++t) invA<N, T>(b.data(), 1, z.data(), 1, t, tw.data());
    // permuted order: forward stage B in place, read through perm_pos
    std::vector<cplx<T>> q = a;
    for (int k1 = 0; k1 < N1; ++k1) fwdB<N, false, T>(q.data(), 1, q.data(), 1, k1, tw.data());
    for (int k = 0; k < N; ++k) p[k] = q[perm_pos<N>(k)];
    std::fprintf(f, "%d %d\n", N, (int)sizeof(T));
    for (int j = 0; j < N; ++j)
        std::fprintf(f, "%.17g %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", (double)x[j].x, (double)x[j].y,
                     (double)y[j].x, (double)y[j].y, (double)z[j].x, (double)z[j].y, (double)p[j].x,
                     (double)p[j].y);
}

int main() {
#define RUN(n) run<n, double>(stdout); run<n, float>(stdout);
    RUN(3) RUN(5) RUN(9) RUN(15) RUN(25) RUN(27) RUN(45) RUN(75) RUN(81) RUN(125) RUN(135) RUN(225) RUN(243)
    return 0;
}
"""


def _cxx():
    return shutil.which("g++") or shutil.which("c++")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = _cxx()
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("fftcore")
    (d / "cuda_runtime.h").write_text(STUB)
    (d / "harness.cpp").write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", str(d), "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    str(d / "harness.cpp"), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    res, i = {}, 0
    while i < len(out) and out[i].strip():
        N, size = map(int, out[i].split())
        rows = np.array([[float(v) for v in out[i + 1 + j].split()] for j in range(N)])
        res[(N, size)] = rows
        i += N + 1
    return res


@pytest.mark.parametrize("N", GRIDS)
@pytest.mark.parametrize("size", [8, 4])
def test_pencil_fft_matches_numpy(results, N, size):
    r = results[(N, size)]
    x = r[:, 0] + 1j * r[:, 1]
    y = r[:, 2] + 1j * r[:, 3]
    z = r[:, 4] + 1j * r[:, 5]
    p = r[:, 6] + 1j * r[:, 7]
    ref = np.fft.fft(x)
    tol = 1e-14 if size == 8 else 2e-6
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= tol * scale * np.log2(N + 1)          # forward, natural order
    assert np.abs(p - ref).max() <= tol * scale * np.log2(N + 1)          # forward, permuted order
    assert np.abs(z - N * x).max() <= tol * N * np.abs(x).max() * np.log2(N + 1) * 2  # inverse
