// The autotuner's schedule variants of the FP32 CG passes for one grid size
// (compiled once per supported N with -DFFTG_N=<N>, like passes_inst.cu).
#include "schedule.cuh"

#ifndef FFTG_N
#error "compile with -DFFTG_N=<grid size>"
#endif

namespace fftg {
template cudaError_t run_variant_n<FFTG_N>(int, int, const PassArgs&, int, cudaStream_t);
template VariantShape variant_shape_n<FFTG_N>(int, int);
}
