// The macroscale bar of the multiscale diffusion (Sec. 3.2) on the device:
// nodal macro concentrations c_m (m = 0 .. M) of a bar along X whose face
// X = 0 takes a constant influx and whose far end is closed; element e
// (nodes e, e + 1) carries RVE e of a batched context at its midpoint.
//   k_bar_inputs: grad c_mac = ((c_{e+1} - c_e) / dX, 0, 0) and
//                 c_macro = (c_e + c_{e+1}) / 2 of every element, the
//                 per-problem inputs of the RVEs' homogenised diffusion;
//   k_bar_update: forward Euler on the lumped finite-difference scheme,
//                 c_m += dt / w_m (J_{m-1/2} - J_{m+1/2}) with w = dX inside,
//                 dX / 2 at the ends, J_{e+1/2} = <j_x> of RVE e (read from
//                 the diffusion statistics the step left on the device),
//                 J_{-1/2} = the influx, J_{M+1/2} = 0.
// The bar has M + 1 values: both kernels are one block.
#include "fftmech_internal.cuh"

namespace fftmech {

static constexpr int kBarThreads = 256;

__global__ void k_bar_inputs(int M, double dX, const double* __restrict__ c, double* __restrict__ cbar,
                             double* __restrict__ G) {
  for (int e = threadIdx.x; e < M; e += blockDim.x) {
    G[3 * e] = (c[e + 1] - c[e]) / dX;
    G[3 * e + 1] = 0.0;
    G[3 * e + 2] = 0.0;
    cbar[e] = 0.5 * (c[e] + c[e + 1]);
  }
}

// res: per-problem diffusion statistics, `stride` doubles each, <j_x> at 2.
__global__ void k_bar_update(int M, double dX, double dt, double flux_in, double* __restrict__ c,
                             const double* __restrict__ res, int stride) {
  for (int m = threadIdx.x; m <= M; m += blockDim.x) {
    const double Jl = m == 0 ? flux_in : res[(size_t)(m - 1) * stride + 2];
    const double Jr = m == M ? 0.0 : res[(size_t)m * stride + 2];
    const double w = (m == 0 || m == M) ? 0.5 * dX : dX;
    c[m] += dt / w * (Jl - Jr);
  }
}

cudaError_t launch_bar_inputs(int M, double dX, const double* c, double* cbar, double* G, cudaStream_t st) {
  k_bar_inputs<<<1, kBarThreads, 0, st>>>(M, dX, c, cbar, G);
  return cudaGetLastError();
}

cudaError_t launch_bar_update(int M, double dX, double dt, double flux_in, double* c, const double* res, int stride,
                              cudaStream_t st) {
  k_bar_update<<<1, kBarThreads, 0, st>>>(M, dX, dt, flux_in, c, res, stride);
  return cudaGetLastError();
}

}  // namespace fftmech
