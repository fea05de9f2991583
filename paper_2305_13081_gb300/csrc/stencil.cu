// Split-iteration stencil kernels (q = K p, <p, K p>) for both precisions.
#include "stencil.cuh"

namespace fftmech {
#define FFTMECH_INST_STEN(T)                                                                            \
  template cudaError_t launch_sten2<T, 1>(const Op<T>&, const Vec2<T>&, const StenShape&, cudaStream_t); \
  template cudaError_t launch_sten2<T, 2>(const Op<T>&, const Vec2<T>&, const StenShape&, cudaStream_t); \
  template cudaError_t launch_sten3<T, 1>(const Op<T>&, const Vec2<T>&, const StenShape&, cudaStream_t); \
  template cudaError_t launch_sten3<T, 3>(const Op<T>&, const Vec2<T>&, const StenShape&, cudaStream_t);
FFTMECH_INST_STEN(float)
FFTMECH_INST_STEN(double)
}  // namespace fftmech
