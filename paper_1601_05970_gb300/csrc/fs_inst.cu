// Finite-strain pass kernels of one grid size, compiled once for each
// supported N with -DFFTG_N=<N> (in parallel with the other units).
#include "fs_passes.cuh"

#ifndef FFTG_N
#error "compile with -DFFTG_N=<grid size>"
#endif

namespace fftg {
template cudaError_t run_fs_pass_n<FFTG_N>(FsPassKind, const FsArgs&, cudaStream_t);
}
