// Split-iteration x-line kernels (and the fused direction-stencil kernel) for lines of 128 points (compile-time FFT, float).
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(128)
FFTMECH_INST_XDS_FIXED(128)
}  // namespace fftmech
