"""fftg: GB300-native FFT-Galerkin Newton-CG micromechanics (arXiv:1601.05970).

The solver runs in the CUDA kernels of libfftg.so (C-ABI in include/fftg.h);
`paper_1601_05970_gb300.fftg` is its thin Python binding and
`paper_1601_05970_gb300.inputs` the seeded synthetic inputs.
"""
