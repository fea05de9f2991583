// 2D PCG kernels instantiated for the FAM_9 radix family.
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_FAMILY(FAM_9)
}  // namespace fftmech
