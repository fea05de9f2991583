// 3D PCG kernels instantiated for the FAM_9 radix family.
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_FAMILY(FAM_9)
}  // namespace fftmech
