// Split-iteration x-line kernels instantiated for the FAM_ALL radix family.
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_ALL)
FFTMECH_INST_LINES_T(double, FAM_ALL)
}  // namespace fftmech
