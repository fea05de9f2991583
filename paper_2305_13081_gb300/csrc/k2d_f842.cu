// 2D PCG kernels instantiated for the FAM_842 radix family.
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_FAMILY(FAM_842)
}  // namespace fftmech
