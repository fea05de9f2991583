// 3D PCG kernels instantiated for the FAM_842 radix family.
#include "kernels3d.cuh"

namespace fftmech {
FFTMECH_INST3_FAMILY(FAM_842)
}  // namespace fftmech
