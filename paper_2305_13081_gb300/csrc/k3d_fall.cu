// 3D PCG kernels instantiated for the FAM_ALL radix family.
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_FAMILY(FAM_ALL)
}  // namespace fftmech
