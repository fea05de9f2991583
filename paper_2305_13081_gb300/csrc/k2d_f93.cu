// 2D PCG kernels instantiated for the FAM_93 radix family.
#include "kernels2d.cuh"

namespace fftmech {
FFTMECH_INST_FAMILY(FAM_93)
}  // namespace fftmech
