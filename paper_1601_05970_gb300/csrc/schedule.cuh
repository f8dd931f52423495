// Schedules of the FP32 passes of the mixed CG iteration, chosen at run time
// by the autotuner (autotune.cu): per grid size and pass, one of
// kVariants (radix split, tile) pairs. Variant 0 is the default schedule
// compiled into run_pass_n; variants 1 .. kVariants-1 are instantiated per
// grid size in passes_tune.cu.
//
//   P1 (x3, rows), P5 (x3, rows): 0 default; 1 the other radix split;
//                                 2 half the rows per block; 3 twice the rows
//   P2, P4 (x2, columns):         0 default; 1 the other radix split;
//                                 2 32 columns per block; 3 both
//   P3 (x1 + Ghat, columns):      0 default; 1 the other radix split;
//                                 2 half the columns per block;
//                                 3 the default tile with stage B, Ghat
//                                   and the inverse stage B in one phase
//                                   (k_p3f; splits with 1 < N2 <= 9, else
//                                   the default)
//
// A schedule changes only how the same transforms are split into register
// DFTs and how pencils are grouped into blocks: the results agree to FP32
// rounding.
#pragma once

#include <algorithm>

#include "passes.cuh"

namespace fftg {

enum : int { TK_P1 = 0, TK_P2 = 1, TK_P3 = 2, TK_P4 = 3, TK_P5 = 4, TK_COUNT = 5 };
constexpr int kVariants = 4;

// The other radix split of N: the default's two factors swapped, or for a
// single-stage default (N <= 27) a two-stage split; N itself when there is
// none.
template <int N>
struct AltSplit {
    static constexpr int A = Plan<N>::N2 > 1 ? Plan<N>::N2
                             : (N % 9 == 0 && N > 9) ? 9
                             : (N % 5 == 0 && N > 5) ? 5
                             : (N % 3 == 0 && N > 3) ? 3
                                                     : N;
};

template <int N, int TK, int V>
struct VariantOf {
    static constexpr bool cols = TK == TK_P2 || TK == TK_P4;
    static constexpr bool fused = TK == TK_P3 && V == 3;
    static constexpr int A = (V == 1 || (V == 3 && cols)) ? AltSplit<N>::A : Plan<N>::N1;
    static constexpr int TV = V == 0 ? 0 : V == 1 ? 0 : V == 2 ? 1 : cols ? 1 : fused ? 0 : 2;
};

template <int N, int TK, int V>
cudaError_t launch_variant(const PassArgs& a, int nf, cudaStream_t s) {
    using VO = VariantOf<N, TK, V>;
    using C = Cfg<N, float, VO::A, VO::TV>;
    if constexpr (TK == TK_P1) {
        return launch_k(k_p1<N, float, P1_CGF, VO::A, VO::TV>, dim3(C::row_blocks, 1, nf), C::smem_rows, a, s);
    } else if constexpr (TK == TK_P5) {
        return launch_k(k_p5<N, float, P5_CGF, float, VO::A, VO::TV>, dim3(C::row_blocks, 1, nf), C::smem_rows,
                        a, s);
    } else if constexpr (TK == TK_P3 && VO::fused && P3f<N, VO::A>::ok) {
        return launch_k(k_p3f<N, VO::A>, dim3((C::H + C::W3 - 1) / C::W3, N, nf), C::smem_p3, a, s,
                        P3f<N, VO::A>::NT);
    } else if constexpr (TK == TK_P3) {
        return launch_k(k_p3<N, float, VO::A, VO::TV>, dim3((C::H + C::W3 - 1) / C::W3, N, nf), C::smem_p3, a, s,
                        C::T3);
    } else {
        const dim3 g((C::H + C::W2 - 1) / C::W2, (6 * N + C::S2 - 1) / C::S2, nf);
        return launch_k(k_p24<N, float, TK == TK_P2, 6, VO::A, VO::TV>, g, C::smem_p24, a, s, C::T2);
    }
}

// Variants 1 .. kVariants-1 of the tuned kinds at grid N (passes_tune.cu).
template <int N>
cudaError_t run_variant_n(int tk, int v, const PassArgs& a, int nf, cudaStream_t s) {
    switch (tk * kVariants + v) {
#define FFTG_VAR(tk_, v_) \
    case tk_ * kVariants + v_: return launch_variant<N, tk_, v_>(a, nf, s);
        FFTG_VAR(TK_P1, 1) FFTG_VAR(TK_P1, 2) FFTG_VAR(TK_P1, 3)
        FFTG_VAR(TK_P2, 1) FFTG_VAR(TK_P2, 2) FFTG_VAR(TK_P2, 3)
        FFTG_VAR(TK_P3, 1) FFTG_VAR(TK_P3, 2) FFTG_VAR(TK_P3, 3)
        FFTG_VAR(TK_P4, 1) FFTG_VAR(TK_P4, 2) FFTG_VAR(TK_P4, 3)
        FFTG_VAR(TK_P5, 1) FFTG_VAR(TK_P5, 2) FFTG_VAR(TK_P5, 3)
#undef FFTG_VAR
        default: return cudaErrorInvalidValue;
    }
}

// Block geometry of a variant, for the host (partial-sum buffers and the
// tuner's description of each schedule).
struct VariantShape {
    int n1, n2;     // radix split
    int rows;       // P1/P5 rows per block
    int cols;       // P3 or P2/P4 columns per block
    int blocks;     // blocks per field
};

template <int N, int TK, int V>
VariantShape shape_of() {
    using VO = VariantOf<N, TK, V>;
    using C = Cfg<N, float, VO::A, VO::TV>;
    VariantShape sh{VO::A, N / VO::A, C::R, TK == TK_P3 ? C::W3 : C::W2, 0};
    if (TK == TK_P1 || TK == TK_P5)
        sh.blocks = C::row_blocks;
    else if (TK == TK_P3)
        sh.blocks = ((C::H + C::W3 - 1) / C::W3) * N;
    else
        sh.blocks = ((C::H + C::W2 - 1) / C::W2) * ((6 * N + C::S2 - 1) / C::S2);
    return sh;
}

template <int N>
VariantShape variant_shape_n(int tk, int v) {
    switch (tk * kVariants + v) {
#define FFTG_SHAPE(tk_, v_) \
    case tk_ * kVariants + v_: return shape_of<N, tk_, v_>();
        FFTG_SHAPE(TK_P1, 0) FFTG_SHAPE(TK_P1, 1) FFTG_SHAPE(TK_P1, 2) FFTG_SHAPE(TK_P1, 3)
        FFTG_SHAPE(TK_P2, 0) FFTG_SHAPE(TK_P2, 1) FFTG_SHAPE(TK_P2, 2) FFTG_SHAPE(TK_P2, 3)
        FFTG_SHAPE(TK_P3, 0) FFTG_SHAPE(TK_P3, 1) FFTG_SHAPE(TK_P3, 2) FFTG_SHAPE(TK_P3, 3)
        FFTG_SHAPE(TK_P4, 0) FFTG_SHAPE(TK_P4, 1) FFTG_SHAPE(TK_P4, 2) FFTG_SHAPE(TK_P4, 3)
        FFTG_SHAPE(TK_P5, 0) FFTG_SHAPE(TK_P5, 1) FFTG_SHAPE(TK_P5, 2) FFTG_SHAPE(TK_P5, 3)
#undef FFTG_SHAPE
        default: return VariantShape{0, 0, 0, 0, 0};
    }
}

// Host side (autotune.cu): the variant in use for (N, tuned kind), 0 unless
// a schedule was set or tuned; -1 for kinds that are not tuned.
int tuned_kind(int pass_kind);
int schedule_variant(int N, int tk);
cudaError_t run_variant(int N, int tk, int v, const PassArgs& a, int nf, cudaStream_t s);
VariantShape variant_shape(int N, int tk, int v);

}  // namespace fftg
