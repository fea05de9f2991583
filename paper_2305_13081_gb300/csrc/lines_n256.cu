// Split-iteration x-line kernels (and the fused direction-stencil kernel) for lines of 256 points (compile-time FFT, float).
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(256)
FFTMECH_INST_XDS_FIXED(256)
}  // namespace fftmech
