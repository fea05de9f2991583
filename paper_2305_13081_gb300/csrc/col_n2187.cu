// 2D column passes for columns of 2187 points (compile-time FFT, float).
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(2187)
}  // namespace fftmech
