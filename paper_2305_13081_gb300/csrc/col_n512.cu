// 2D column passes for columns of 512 points (compile-time FFT, float).
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_COL_FIXED(512)
}  // namespace fftmech
