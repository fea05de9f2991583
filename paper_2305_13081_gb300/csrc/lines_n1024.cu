// Split-iteration x-line kernels for lines of 1024 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(1024)
}  // namespace fftmech
