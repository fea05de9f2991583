// Pointwise kernels of the reverse sweep of the staggered solve (the
// discrete adjoint of Algorithm 1 with a prescribed, ramped eigenstrain; an
// extension, the paper solves forward only). The two linear solves of a
// reverse step (phase-field adjoint, equilibrium adjoint) run on the
// library's PCG; these kernels connect them:
//   k_adj_m0b:     m0 = a + <H> of the phase-field preconditioner;
//   k_adj_history: phase-field adjoint -> history max -> psi+ of Eq. (energy):
//                  dJ/dH, the equilibrium adjoint's right-hand side
//                  tau = dJ/dpsi dpsi/deps_el and the explicit dJ/de_s;
//   k_adj_eqpost:  equilibrium adjoint mu -> dJ/de_s (through the load) and
//                  dJ/dd_{s-1} (through the degradation), accumulated into
//                  the gradient with the ramp factor of the step;
//   k_absmax / k_apply_scale: a right-hand side scaled by a power of two to
//                  the magnitude of the forward solve's, the reciprocal kept
//                  on the device for the solution. The adjoint's right-hand
//                  sides carry the voxel volume h^d (1e-16 in 3D at h = 5 um);
//                  unscaled, the float residual products r.M^-1 r fall out of
//                  float's normal range before the tolerance is reached.
//                  Power-of-two scaling is exact, so the FP64 path computes
//                  the same numbers as without it.
#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

static constexpr int kAdjThreads = 256;

static inline int adj_grid(long long n) {
  long long g = (n + kAdjThreads - 1) / kAdjThreads;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

// m0b[0] = a + mean(H) (one problem), one block.
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) k_adj_m0b(long long N, const T* H, double a, double* m0b) {
  __shared__ double red[32];
  double acc[1] = {0.0};
  for (long long i = threadIdx.x; i < N; i += blockDim.x) acc[0] += (double)H[i];
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) m0b[0] = a + acc[0] / (double)N;
}

// Voigt slot layout: 2D xx, yy, xy; 3D xx, yy, zz, yz, xz, xy.
template <int DIM>
struct Voigt;
template <>
struct Voigt<2> {
  static constexpr int NV = 3;
  static __device__ __forceinline__ bool diag(int k) { return k < 2; }
};
template <>
struct Voigt<3> {
  static constexpr int NV = 6;
  static __device__ __forceinline__ bool diag(int k) { return k < 3; }
};

// Per voxel of step s (e_s = scale e(x), strain eps_s, H_{s-1}, d_s, the
// phase-field adjoint lam_pf solved for dJ/dd_s):
//   dJ/dH_s = dJ_dH + (1 - d_s) lam_pf;
//   psi+ = psi+(eps_s - e_s I) recomputed as the forward's history kernel
//   does; where psi+ >= H_{s-1} the history took psi+: dJ/dpsi = dJ/dH_s
//   and dJ_dH (the part that reaches H_{s-1}) = 0, else dJ/dpsi = 0;
//   tau = dJ/dpsi (K [tr]_+ I + 2 mu dev eps_el)  (Voigt, tensor shear);
//   dJde = -dJ/dpsi d K [tr]_+;
//   last step of the energy objective: dJde -= tr(sigma) h^d and
//   ddirect = 1/2 g'(d_{s-1}) eps_el : C : eps_el h^d (else 0).
template <typename T, int DIM>
__global__ void k_adj_history(long long N, const uint8_t* __restrict__ phase, double lam0, double lam1, double mu0,
                              double mu1, const T* __restrict__ strain, const T* __restrict__ efield, double scale,
                              const T* __restrict__ Hprev, const double* __restrict__ d, const double* lam_pf,
                              const double* lam_inv, double* dJ_dH, T* tau, double* dJde, double* ddirect,
                              int energy_last, const double* __restrict__ dprev, double kappa, double vol) {
  using V = Voigt<DIM>;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const bool sol = phase[i] != 0;
    const double lam = sol ? lam1 : lam0, mu = sol ? mu1 : mu0;
    const double e = (double)(T)(scale * (double)efield[i]);  // as the forward step stored it
    double el[6];
#pragma unroll
    for (int k = 0; k < V::NV; ++k) el[k] = (double)strain[k * N + i] - (V::diag(k) ? e : 0.0);
    double psi, tr;
    double dv[6];
    if constexpr (DIM == 2) {
      tr = el[0] + el[1];
      const double dx = el[0] - 0.5 * tr, dy = el[1] - 0.5 * tr;
      const double trp = tr > 0 ? tr : 0.0;
      psi = 0.5 * (lam + mu) * trp * trp + mu * (dx * dx + dy * dy + 2 * el[2] * el[2]);
      dv[0] = dx;
      dv[1] = dy;
      dv[2] = el[2];
    } else {
      tr = el[0] + el[1] + el[2];
      const double dx = el[0] - tr / 3.0, dy = el[1] - tr / 3.0, dz = el[2] - tr / 3.0;
      const double trp = tr > 0 ? tr : 0.0;
      const double K3 = lam + 2.0 * mu / 3.0;
      psi = 0.5 * K3 * trp * trp + mu * (dx * dx + dy * dy + dz * dz + 2 * (el[5] * el[5] + el[4] * el[4] + el[3] * el[3]));
      dv[0] = dx;
      dv[1] = dy;
      dv[2] = dz;
      dv[3] = el[3];
      dv[4] = el[4];
      dv[5] = el[5];
    }
    double total = dJ_dH[i] + (lam_pf ? (1.0 - d[i]) * (lam_pf[i] * lam_inv[0]) : 0.0);
    const bool take = psi >= (double)Hprev[i];
    const double dpsi = take ? total : 0.0;
    dJ_dH[i] = take ? 0.0 : total;
    const double K = lam + 2.0 * mu / DIM;
    const double trp = tr > 0 ? tr : 0.0;
#pragma unroll
    for (int k = 0; k < V::NV; ++k) tau[k * N + i] = (T)(dpsi * ((V::diag(k) ? K * trp : 0.0) + 2.0 * mu * dv[k]));
    double de = -dpsi * DIM * K * trp;
    double dd = 0.0;
    if (energy_last) {
      const double dp = dprev ? dprev[i] : 0.0;
      const double g = (1.0 - dp) * (1.0 - dp) + kappa;
      const double gp = -2.0 * (1.0 - dp);
      // C : eps_el (undegraded) and eps_el : C : eps_el (shear counted twice)
      double q = 0.0, trs = 0.0;
#pragma unroll
      for (int k = 0; k < V::NV; ++k) {
        const double c = (V::diag(k) ? lam * tr : 0.0) + 2.0 * mu * el[k];
        q += (V::diag(k) ? 1.0 : 2.0) * c * el[k];
        if (V::diag(k)) trs += c;
      }
      de += -g * trs * vol;
      dd = 0.5 * gp * q * vol;
    }
    dJde[i] = de;
    ddirect[i] = dd;
  }
}

// Per voxel: eps(mu) = sym grad+ mu (periodic forward differences of the
// equilibrium adjoint mu, D = DIM components), then
//   dJde += g(d_{s-1}) (DIM lam + 2 mu) tr eps(mu),
//   dJdd = ddirect - g'(d_{s-1}) (C : eps_el) : eps(mu),
//   grad += scale dJde.
template <typename T, int DIM>
__global__ void k_adj_eqpost(int nx, int ny, int nz, const uint8_t* __restrict__ phase, double lam0, double lam1,
                             double mu0, double mu1, const T* __restrict__ strain, const T* __restrict__ efield,
                             double scale, const double* __restrict__ dprev, double kappa, const double* __restrict__ mu,
                             const double* mu_inv, double h, const double* __restrict__ dJde,
                             const double* __restrict__ ddirect, double* dJdd, double* grad) {
  using V = Voigt<DIM>;
  const long long N = (long long)nx * ny * nz;
  const double ih = mu_inv[0] / h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const long long ixp = i - x + (x + 1 == nx ? 0 : x + 1);
    const long long iyp = i + (long long)((y + 1 == ny ? 0 : y + 1) - y) * nx;
    const long long izp = i + (long long)((z + 1 == nz ? 0 : z + 1) - z) * nx * ny;
    double em[6];
    if constexpr (DIM == 2) {
      const double* ux = mu;
      const double* uy = mu + N;
      em[0] = (ux[ixp] - ux[i]) * ih;
      em[1] = (uy[iyp] - uy[i]) * ih;
      em[2] = 0.5 * ((ux[iyp] - ux[i]) + (uy[ixp] - uy[i])) * ih;
    } else {
      const double* ux = mu;
      const double* uy = mu + N;
      const double* uz = mu + 2 * N;
      em[0] = (ux[ixp] - ux[i]) * ih;
      em[1] = (uy[iyp] - uy[i]) * ih;
      em[2] = (uz[izp] - uz[i]) * ih;
      em[3] = 0.5 * ((uy[izp] - uy[i]) + (uz[iyp] - uz[i])) * ih;
      em[4] = 0.5 * ((ux[izp] - ux[i]) + (uz[ixp] - uz[i])) * ih;
      em[5] = 0.5 * ((ux[iyp] - ux[i]) + (uy[ixp] - uy[i])) * ih;
    }
    const bool sol = phase[i] != 0;
    const double lam = sol ? lam1 : lam0, m = sol ? mu1 : mu0;
    const double e = (double)(T)(scale * (double)efield[i]);
    double el[6], trm = 0.0, tr = 0.0;
#pragma unroll
    for (int k = 0; k < V::NV; ++k) {
      el[k] = (double)strain[k * N + i] - (V::diag(k) ? e : 0.0);
      if (V::diag(k)) {
        trm += em[k];
        tr += el[k];
      }
    }
    const double dp = dprev ? dprev[i] : 0.0;
    const double g = (1.0 - dp) * (1.0 - dp) + kappa;
    const double gp = -2.0 * (1.0 - dp);
    double ce = 0.0;  // (C : eps_el) : eps(mu), shear counted twice
#pragma unroll
    for (int k = 0; k < V::NV; ++k) {
      const double c = (V::diag(k) ? lam * tr : 0.0) + 2.0 * m * el[k];
      ce += (V::diag(k) ? 1.0 : 2.0) * c * em[k];
    }
    const double de = dJde[i] + g * (DIM * lam + 2.0 * m) * trm;
    dJdd[i] = ddirect[i] - gp * ce;
    grad[i] += scale * de;
  }
}

// *m = max |x_i| as the bits of a non-negative double (*m zeroed before).
template <typename X>
__global__ void __launch_bounds__(kAdjThreads) k_absmax(long long n, const X* __restrict__ x, unsigned long long* m) {
  __shared__ double red[kAdjThreads / 32];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v = fmax(v, fabs((double)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kAdjThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMax(m, (unsigned long long)__double_as_longlong(v));
  }
}

// s = 2^k with s max|x| in [target / 2, target) (s = 1 for a zero field);
// x *= s, scale[0] = s, scale[1] = 1 / s.
template <typename X>
__global__ void k_apply_scale(long long n, X* x, const unsigned long long* m, double target, double* scale) {
  const double mx = __longlong_as_double((long long)m[0]);
  double s = 1.0;
  if (mx > 0.0 && isfinite(mx)) {
    int e;
    frexp(target / mx, &e);
    e = max(-1000, min(1000, e - 1));
    s = ldexp(1.0, e);
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = (X)((double)x[i] * s);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scale[0] = s;
    scale[1] = 1.0 / s;
  }
}

template <typename X>
cudaError_t launch_adj_normalise(long long n, X* x, unsigned long long* m, double target, double* scale,
                                 cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(m, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  k_absmax<X><<<adj_grid(n), kAdjThreads, 0, st>>>(n, x, m);
  k_apply_scale<X><<<adj_grid(n), kAdjThreads, 0, st>>>(n, x, m, target, scale);
  return cudaGetLastError();
}
template cudaError_t launch_adj_normalise<float>(long long, float*, unsigned long long*, double, double*, cudaStream_t);
template cudaError_t launch_adj_normalise<double>(long long, double*, unsigned long long*, double, double*,
                                                  cudaStream_t);

__global__ void k_fill(long long N, double v, double* p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_fill(long long N, double v, double* p, cudaStream_t st) {
  k_fill<<<adj_grid(N), kAdjThreads, 0, st>>>(N, v, p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_m0b(long long N, const T* H, double a, double* m0b, cudaStream_t st) {
  k_adj_m0b<T><<<1, kAdjThreads, 0, st>>>(N, H, a, m0b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_history(int dim, long long N, const uint8_t* phase, double lam0, double lam1, double mu0,
                               double mu1, const T* strain, const T* efield, double scale, const T* Hprev,
                               const double* d, const double* lam_pf, const double* lam_inv, double* dJ_dH, T* tau,
                               double* dJde, double* ddirect, int energy_last, const double* dprev, double kappa,
                               double vol, cudaStream_t st) {
  if (dim == 2)
    k_adj_history<T, 2><<<adj_grid(N), kAdjThreads, 0, st>>>(N, phase, lam0, lam1, mu0, mu1, strain, efield, scale,
                                                              Hprev, d, lam_pf, lam_inv, dJ_dH, tau, dJde, ddirect,
                                                              energy_last, dprev, kappa, vol);
  else
    k_adj_history<T, 3><<<adj_grid(N), kAdjThreads, 0, st>>>(N, phase, lam0, lam1, mu0, mu1, strain, efield, scale,
                                                              Hprev, d, lam_pf, lam_inv, dJ_dH, tau, dJde, ddirect,
                                                              energy_last, dprev, kappa, vol);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_eqpost(int dim, int nx, int ny, int nz, const uint8_t* phase, double lam0, double lam1,
                              double mu0, double mu1, const T* strain, const T* efield, double scale,
                              const double* dprev, double kappa, const double* mu, const double* mu_inv, double h,
                              const double* dJde, const double* ddirect, double* dJdd, double* grad,
                              cudaStream_t st) {
  const long long N = (long long)nx * ny * nz;
  if (dim == 2)
    k_adj_eqpost<T, 2><<<adj_grid(N), kAdjThreads, 0, st>>>(nx, ny, 1, phase, lam0, lam1, mu0, mu1, strain, efield,
                                                             scale, dprev, kappa, mu, mu_inv, h, dJde, ddirect, dJdd, grad);
  else
    k_adj_eqpost<T, 3><<<adj_grid(N), kAdjThreads, 0, st>>>(nx, ny, nz, phase, lam0, lam1, mu0, mu1, strain, efield,
                                                             scale, dprev, kappa, mu, mu_inv, h, dJde, ddirect, dJdd, grad);
  return cudaGetLastError();
}

#define FFTMECH_ADJ_INST(T)                                                                                          \
  template cudaError_t launch_adj_m0b<T>(long long, const T*, double, double*, cudaStream_t);                        \
  template cudaError_t launch_adj_history<T>(int, long long, const uint8_t*, double, double, double, double, const T*, \
                                             const T*, double, const T*, const double*, const double*, const double*, \
                                             double*, T*, double*, double*, int, const double*, double, double,      \
                                             cudaStream_t);                                                          \
  template cudaError_t launch_adj_eqpost<T>(int, int, int, int, const uint8_t*, double, double, double, double,      \
                                            const T*, const T*, double, const double*, double, const double*,        \
                                            const double*, double, const double*, const double*, double*, double*,  \
                                            cudaStream_t);
FFTMECH_ADJ_INST(float)
FFTMECH_ADJ_INST(double)

}  // namespace fftmech
