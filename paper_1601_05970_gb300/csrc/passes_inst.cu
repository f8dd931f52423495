// One translation unit per grid size: compiled once for each supported N
// with -DFFTG_N=<N>, so the build of the pass kernels runs in parallel.
#include "passes.cuh"

#ifndef FFTG_N
#error "compile with -DFFTG_N=<grid size>"
#endif

namespace fftg {
template cudaError_t run_pass_n<FFTG_N>(PassKind, const PassArgs&, int, cudaStream_t);
}
