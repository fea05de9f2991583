// Split-iteration x-line kernels for lines of 2187 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(2187)
}  // namespace fftmech
