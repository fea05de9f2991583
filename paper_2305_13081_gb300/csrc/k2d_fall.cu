// 2D PCG kernels instantiated for the FAM_ALL radix family.
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_FAMILY(FAM_ALL)
}  // namespace fftmech
