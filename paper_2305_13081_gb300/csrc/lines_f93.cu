// Split-iteration x-line kernels (and the fused direction-stencil kernel) instantiated for the FAM_93 radix family.
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_93)
FFTMECH_INST_XDS_T(float, FAM_93)
FFTMECH_INST_LINES_T(double, FAM_93)
FFTMECH_INST_XDS_T(double, FAM_93)
}  // namespace fftmech
