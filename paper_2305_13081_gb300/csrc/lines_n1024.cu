// Split-iteration x-line kernels (and the fused direction-stencil kernel) for lines of 1024 points (compile-time FFT, float).
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(1024)
FFTMECH_INST_XDS_FIXED(1024)
}  // namespace fftmech
