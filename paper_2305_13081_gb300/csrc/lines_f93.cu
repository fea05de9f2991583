// Split-iteration x-line kernels instantiated for the FAM_93 radix family.
#include "lines.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_93)
FFTMECH_INST_LINES_T(double, FAM_93)
}  // namespace fftmech
