// 3D y / z line passes for lines of 1024 points (compile-time FFT, float).
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_LINES_FIXED(1024)
}  // namespace fftmech
