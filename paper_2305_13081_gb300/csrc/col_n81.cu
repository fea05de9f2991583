// 2D column passes for columns of 81 points (compile-time FFT, float).
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(81)
}  // namespace fftmech
