// 2D column passes for columns of 1024 points (compile-time FFT, float), Laplace and
// reference-medium preconditioners.
#include "kernels2d.cuh"
#include "colpass_ms.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(1024)
FFTMECH_INST_COL_MS_FIXED(1024)
}  // namespace fftmech
