// 3D PCG kernels instantiated for the FAM_93 radix family.
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_FAMILY(FAM_93)
}  // namespace fftmech
