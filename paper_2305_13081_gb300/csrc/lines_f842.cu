// Split-iteration x-line kernels (and the fused direction-stencil kernel) instantiated for the FAM_842 radix family.
#include "dirsten.cuh"

namespace fftmech {
FFTMECH_INST_LINES_T(float, FAM_842)
FFTMECH_INST_XDS_T(float, FAM_842)
FFTMECH_INST_LINES_T(double, FAM_842)
FFTMECH_INST_XDS_T(double, FAM_842)
}  // namespace fftmech
