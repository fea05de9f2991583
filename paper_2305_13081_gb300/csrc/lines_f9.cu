// Split-iteration x-line kernels (and the fused direction-stencil kernel) instantiated for the FAM_9 radix family.
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_9)
FFTMECH_INST_XDS_T(float, FAM_9)
FFTMECH_INST_LINES_T(double, FAM_9)
FFTMECH_INST_XDS_T(double, FAM_9)
}  // namespace fftmech
