// Split-iteration x-line kernels instantiated for the FAM_842 radix family.
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_842)
FFTMECH_INST_LINES_T(double, FAM_842)
}  // namespace fftmech
