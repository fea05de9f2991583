// Split-iteration x-line kernels for lines of 729 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(729)
}  // namespace fftmech
