// Split-iteration x-line kernels instantiated for the FAM_9 radix family.
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_9)
FFTMECH_INST_LINES_T(double, FAM_9)
}  // namespace fftmech
