// 2D column passes for columns of 256 points (compile-time FFT, float).
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(256)
}  // namespace fftmech
