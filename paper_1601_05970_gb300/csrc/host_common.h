// Host-side helpers shared by the small- and finite-strain drivers.
#pragma once

#include <cmath>

namespace fftg {

// Grid sizes with a compiled plan: odd, 3^a 5^b, up to 243.
inline bool supported_grid(int N) {
    switch (N) {
        case 3: case 5: case 9: case 15: case 25: case 27: case 45: case 75: case 81: case 125:
        case 135: case 225: case 243:
            return true;
        default:
            return false;
    }
}

// Component stride of every field: N^3 rounded up past N^3 + 4 to a
// multiple of 32 elements, so each component starts 128-byte aligned and a
// 16-byte vector that straddles the end of the grid stays in the padding.
inline long long comp_stride(int N) {
    const long long V = (long long)N * N * N;
    return ((V + 4 + 31) / 32) * 32;
}

// w_N^j = exp(-2 pi i j / N), evaluated in long double on the host: FP64,
// FP32 and (when twdd is not null) double-float (hi, lo) pairs, 4 floats
// per twiddle (re.hi, re.lo, im.hi, im.lo).
inline void twiddles(int N, double* tw64, float* tw32, float* twdd = nullptr) {
    const long double two_pi = 6.283185307179586476925286766559L;
    for (int j = 0; j < N; ++j) {
        const long double a = two_pi * (long double)j / (long double)N;
        const long double cl = cosl(a), sl = -sinl(a);
        const double c = (double)cl, s = (double)sl;
        tw64[2 * j] = c;
        tw64[2 * j + 1] = s;
        tw32[2 * j] = (float)c;
        tw32[2 * j + 1] = (float)s;
        if (twdd) {
            const float ch = (float)cl, sh = (float)sl;
            twdd[4 * j] = ch;
            twdd[4 * j + 1] = (float)(cl - (long double)ch);
            twdd[4 * j + 2] = sh;
            twdd[4 * j + 3] = (float)(sl - (long double)sh);
        }
    }
}

}  // namespace fftg
