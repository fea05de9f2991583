// Column pass with the reference-medium preconditioner: dispatch to the
// compile-time-plan variants (instantiated with the other fixed-length
// column passes, col_n*.cu) and the runtime-plan variants (here).
#include "colpass_ms.cuh"

namespace fftmech {

#define FFTMECH_MS_EXTERN(N) extern template cudaError_t launch_colpass_ms<float, FAM_ALL, N> FFTMECH_MS_SIG(float);
FFTMECH_MS_EXTERN(81)
FFTMECH_MS_EXTERN(243)
FFTMECH_MS_EXTERN(729)
FFTMECH_MS_EXTERN(2187)
FFTMECH_MS_EXTERN(128)
FFTMECH_MS_EXTERN(256)
FFTMECH_MS_EXTERN(512)
FFTMECH_MS_EXTERN(1024)
#undef FFTMECH_MS_EXTERN

template <typename T>
cudaError_t launch_colpass_ms_f(int fy, int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp,
                                int CW, int threads, int batch, int mode, double* partials, SolverScalars* sc,
                                int* pmode, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (CW == 4) {
#define FFTMECH_N(NY) \
  launch_colpass_ms<T, FAM_ALL, NY>(nx, ny, S, py, sp, CW, threads, batch, mode, partials, sc, pmode, st)
      FFTMECH_FIXED_SWITCH(ny, FFTMECH_N)
#undef FFTMECH_N
    }
  }
#define FFTMECH_C(F) launch_colpass_ms<T, F, 0>(nx, ny, S, py, sp, CW, threads, batch, mode, partials, sc, pmode, st)
  FFTMECH_FAMILY_SWITCH(fy, FFTMECH_C)
#undef FFTMECH_C
}

template cudaError_t launch_colpass_ms_f<float>(int, int, int, cx<float>*, const FftPlanDev<float>&,
                                                const Spec<float>&, int, int, int, int, double*, SolverScalars*,
                                                int*, cudaStream_t);
template cudaError_t launch_colpass_ms_f<double>(int, int, int, cx<double>*, const FftPlanDev<double>&,
                                                 const Spec<double>&, int, int, int, int, double*, SolverScalars*,
                                                 int*, cudaStream_t);

}  // namespace fftmech
