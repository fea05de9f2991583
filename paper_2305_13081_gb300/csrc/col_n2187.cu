// 2D column passes for columns of 2187 points (compile-time FFT, float), Laplace and
// reference-medium preconditioners.
#include "kernels2d.cuh"
#include "colpass_ms.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(2187)
FFTMECH_INST_COL_MS_FIXED(2187)
}  // namespace fftmech
