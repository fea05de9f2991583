// Split-iteration x-line kernels for lines of 243 points (compile-time FFT, float).
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_FIXED(243)
}  // namespace fftmech
