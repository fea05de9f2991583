// 3D y / z line passes for lines of 128 points (compile-time FFT, float).
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_LINES_FIXED(128)
}  // namespace fftmech
