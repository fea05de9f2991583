// 3D y / z line passes for lines of 256 points (compile-time FFT, float).
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_LINES_FIXED(256)
}  // namespace fftmech
