// 2D column passes for columns of 256 points (compile-time FFT, float), Laplace and
// reference-medium preconditioners.
#include "kernels2d.cuh"
#include "colpass_ms.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(256)
FFTMECH_INST_COL_MS_FIXED(256)
}  // namespace fftmech
