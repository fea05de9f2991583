// Split-iteration x-line kernels for lines of 256 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(256)
}  // namespace fftmech
