// Split-iteration x-line kernels for lines of 128 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(128)
}  // namespace fftmech
