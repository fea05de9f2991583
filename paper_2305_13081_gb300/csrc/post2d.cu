// Pointwise physics and FP64 post-processing reductions (2D).
#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

static constexpr int kPostThreads = 256;

static inline int post_grid(long long n) {
  long long g = (n + kPostThreads - 1) / kPostThreads;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

// strain = E + sym grad+ u, stress = g C : (strain - e I) (Eq. solid);
// per problem (blockIdx.y) sums of stress, strain and the energy density
// 1/2 (strain - e I) : stress -> results[b * 7 + k].
template <typename T>
__global__ void k_el_output(Op<T> op, const double* __restrict__ u, T* strain, T* stress,
                            double* partials, double* results, SolverScalars* sc) {
  __shared__ double red[32 * 7];
  const int nx = op.nx, ny = op.ny;
  const long long N = (long long)nx * ny;
  const int b = blockIdx.y;
  const size_t o1 = (size_t)b * N;
  u += 2 * o1;
  if (strain) strain += 3 * o1;
  if (stress) stress += 3 * o1;
  const uint8_t* phase = op.phase + o1;
  const T* g = op.g ? op.g + o1 : nullptr;
  const T* eig = op.eig ? op.eig + o1 : nullptr;
  partials += (size_t)b * gridDim.x * 7;
  const double ih = 1.0 / op.h;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(gi / nx), x = (int)(gi - (long long)y * nx);
    const long long ixp = (long long)y * nx + (x + 1 == nx ? 0 : x + 1);
    const long long iyp = (long long)(y + 1 == ny ? 0 : y + 1) * nx + x;
    const double exx = op.E[0] + (u[ixp] - u[gi]) * ih;
    const double eyy = op.E[1] + (u[N + iyp] - u[N + gi]) * ih;
    const double exy = op.E[2] + 0.5 * ((u[iyp] - u[gi]) + (u[N + ixp] - u[N + gi])) * ih;
    const double e = eig ? (double)eig[gi] : 0.0;
    const int ph = phase[gi] ? 1 : 0;
    const double gg = g ? (double)g[gi] : 1.0;
    const double lam = gg * op.lam[ph], mu = gg * op.mu[ph];
    const double axx = exx - e, ayy = eyy - e;
    const double tr = axx + ayy;
    const double sxx = lam * tr + 2 * mu * axx, syy = lam * tr + 2 * mu * ayy, sxy = 2 * mu * exy;
    if (strain) { strain[gi] = (T)exx; strain[N + gi] = (T)eyy; strain[2 * N + gi] = (T)exy; }
    if (stress) { stress[gi] = (T)sxx; stress[N + gi] = (T)syy; stress[2 * N + gi] = (T)sxy; }
    acc[0] += sxx; acc[1] += syy; acc[2] += sxy;
    acc[3] += exx; acc[4] += eyy; acc[5] += exy;
    acc[6] += 0.5 * (axx * sxx + ayy * syy + 2 * exy * sxy);
  }
  block_sum<7>(acc, red);
  if (publish_partials<7>(acc, partials, &sc[b].cnt[2])) {
    double tot[7];
    gather_partials<7>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 7; ++k) results[b * 7 + k] = tot[k];
  }
}

// Phase statistics of the homogenised diffusion solution (Eq. psi-two-values)
// and the mean flux; the last block of each problem turns them into
// beta_pore, beta_solid. results[b * 6 + .]: beta_pore, beta_solid, <jx>,
// <jy>, porosity, c_macro of the problem.
template <typename T>
__global__ void k_diff_stats(Op<T> op, const double* __restrict__ phi, double hdiff,
                             double c_macro, double* partials, double* results, SolverScalars* sc) {
  __shared__ double red[32 * 10];
  const int nx = op.nx, ny = op.ny;
  const long long N = (long long)nx * ny;
  const int b = blockIdx.y;
  phi += (size_t)b * N;
  const uint8_t* phase = op.phase + (size_t)b * N;
  partials += (size_t)b * gridDim.x * 10;
  const double ih = 1.0 / hdiff;
  const double G0 = macro_grad(op, b, 0), G1 = macro_grad(op, b, 1);
  if (op.cmp) c_macro = op.cmp[b];
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(gi / nx), x = (int)(gi - (long long)y * nx);
    const long long ixp = (long long)y * nx + (x + 1 == nx ? 0 : x + 1);
    const long long iyp = (long long)(y + 1 == ny ? 0 : y + 1) * nx + x;
    const int s = phase[gi] ? 1 : 0;  // 0 pore, 1 solid
    const double ramp = G0 * (x * hdiff) + G1 * (y * hdiff);
    acc[s] += 1.0;
    acc[2 + s] += phi[gi];
    acc[4 + s] += ramp;
    const double D = op.kap[s];
    acc[6] += -D * (G0 + (phi[ixp] - phi[gi]) * ih);
    acc[7] += -D * (G1 + (phi[iyp] - phi[gi]) * ih);
  }
  block_sum<10>(acc, red);
  if (publish_partials<10>(acc, partials, &sc[b].cnt[2])) {
    double tot[10];
    gather_partials<10>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0) {
      const double np = tot[0], ns = tot[1];
      const double eta = np / (double)N;
      double* r = results + b * 6;
      r[0] = np > 0 ? c_macro / eta - (tot[4] + tot[2]) / np : 0.0;
      r[1] = ns > 0 ? -(tot[5] + tot[3]) / ns : 0.0;
      r[2] = tot[6] / (double)N;
      r[3] = tot[7] / (double)N;
      r[4] = eta;
      r[5] = c_macro;
    }
  }
}

// c = grad c_mac . x + phi + beta_phase (Eqs. concentration, concentration-correct),
// beta of problem b from results[b * 6 + 0 / 1]; Gp: per-problem gradients
// (NULL: G0, G1 for all).
__global__ void k_diff_write_c(int nx, int ny, long long total, const uint8_t* __restrict__ phase,
                               const double* __restrict__ phi, double hdiff, double G0, double G1,
                               const double* __restrict__ Gp, const double* __restrict__ beta,
                               double* __restrict__ c) {
  const long long N = (long long)nx * ny;
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
       gi += (long long)gridDim.x * blockDim.x) {
    const long long b = gi / N, li = gi - b * N;
    const int y = (int)(li / nx), x = (int)(li - (long long)y * nx);
    const double bt = phase[gi] ? beta[b * 6 + 1] : beta[b * 6 + 0];
    const double g0 = Gp ? Gp[3 * b] : G0, g1 = Gp ? Gp[3 * b + 1] : G1;
    c[gi] = g0 * (x * hdiff) + g1 * (y * hdiff) + phi[gi] + bt;
  }
}

// H = max(H, psi+(eps - e I)) with Eq. (energy) in 2D; Hd = H as double;
// per problem, m0b[b] = a + mean(H) (the phase-field preconditioner).
template <typename T>
__global__ void k_history(long long N, const uint8_t* __restrict__ phase, double lam0, double lam1,
                          double mu0, double mu1, const T* __restrict__ strain,
                          const T* __restrict__ eig, T* H, double* Hd, double a, double* m0b,
                          double* partials, SolverScalars* sc) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t o1 = (size_t)b * N;
  phase += o1;
  strain += 3 * o1;
  if (eig) eig += o1;
  H += o1;
  Hd += o1;
  partials += (size_t)b * gridDim.x;
  double acc[1] = {0.0};
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const bool sol = phase[gi] != 0;
    const double lam = sol ? lam1 : lam0, mu = sol ? mu1 : mu0;
    const double e = eig ? (double)eig[gi] : 0.0;
    const double exx = (double)strain[gi] - e, eyy = (double)strain[N + gi] - e;
    const double exy = (double)strain[2 * N + gi];
    const double tr = exx + eyy;
    const double dx = exx - 0.5 * tr, dy = eyy - 0.5 * tr;
    const double trp = tr > 0 ? tr : 0.0;
    const double psi = 0.5 * (lam + mu) * trp * trp + mu * (dx * dx + dy * dy + 2 * exy * exy);
    const double h = (double)(T)fmax((double)H[gi], psi);
    H[gi] = (T)h;
    Hd[gi] = h;
    acc[0] += h;
  }
  block_sum<1>(acc, red);
  if (publish_partials<1>(acc, partials, &sc[b].cnt[2])) {
    double tot[1];
    gather_partials<1>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0) m0b[b] = a + tot[0] / (double)N;
  }
}

// Per problem: results[b * 3 + .] = sum d, solid voxels with d > 0.9,
// solid voxels; if m1b, also m1b[b] = (eta D_pore + (1 - eta) D_solid) ih2,
// the mean-diffusivity coefficient of the transient preconditioner.
__global__ void k_pf_stats(long long N, const uint8_t* __restrict__ phase, const double* __restrict__ d,
                           double* partials, double* results, SolverScalars* sc, double Dp, double Ds,
                           double ih2, double* m1b) {
  __shared__ double red[32 * 3];
  const int b = blockIdx.y;
  phase += (size_t)b * N;
  if (d) d += (size_t)b * N;
  partials += (size_t)b * gridDim.x * 3;
  double acc[3] = {0, 0, 0};
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const double v = d ? d[gi] : 0.0;
    acc[0] += v;
    if (phase[gi]) {
      acc[2] += 1.0;
      if (v > 0.9) acc[1] += 1.0;
    }
  }
  block_sum<3>(acc, red);
  if (publish_partials<3>(acc, partials, &sc[b].cnt[2])) {
    double tot[3];
    gather_partials<3>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0) {
      for (int k = 0; k < 3; ++k) results[b * 3 + k] = tot[k];
      if (m1b) {
        const double eta = 1.0 - tot[2] / (double)N;
        m1b[b] = (eta * Dp + (1.0 - eta) * Ds) * ih2;
      }
    }
  }
}

// g(d) = (1 - d)^2 + kappa (Sec. 2.4).
template <typename T>
__global__ void k_degradation(long long N, const double* __restrict__ d, double kappa, T* g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = 1.0 - d[i];
    g[i] = (T)(a * a + kappa);
  }
}

// c_ppt = (c - S)_+ and e = (c_ppt M - 1)_+ in the pores, 0 in the solid (Sec. 2.2).
template <typename T>
__global__ void k_precipitate(long long N, const uint8_t* __restrict__ phase, const double* __restrict__ c,
                              double S, double M, T* c_ppt, T* eig) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double cp = 0.0, e = 0.0;
    if (!phase[i]) {
      cp = c[i] - S;
      cp = cp > 0 ? cp : 0.0;
      e = cp * M - 1.0;
      e = e > 0 ? e : 0.0;
    }
    if (c_ppt) c_ppt[i] = (T)cp;
    eig[i] = (T)e;
  }
}

template <typename T>
__global__ void k_scale_copy(long long N, const T* __restrict__ src, double s, T* dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (T)(s * (double)src[i]);
}

__global__ void k_set_masked(long long N, const uint8_t* __restrict__ mask, double value, double* c) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    if (mask[i]) c[i] = value;
}

template <typename T>
__global__ void k_to_real(long long N, const double* __restrict__ src, T* dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// Double iterate <-> float pair (hi = round(u), lo = round(u - hi)).
__global__ void k_df_split(long long n, const double* __restrict__ u, float* uh, float* ul) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double x = u[i];
    const float h = (float)x;
    uh[i] = h;
    ul[i] = (float)(x - (double)h);
  }
}
__global__ void k_df_merge(long long n, const float* __restrict__ uh, const float* __restrict__ ul,
                           double* u) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = (double)uh[i] + (double)ul[i];
}

// ---------------------------------------------------------------- launchers
static inline dim3 post_grid_b(long long n, int batch) {
  long long g = (n + kPostThreads - 1) / kPostThreads;
  const long long cap = batch > 1 ? 512 : 4096;
  if (g > cap) g = cap;
  return dim3((unsigned)(g < 1 ? 1 : g), (unsigned)batch);
}

template <typename T>
cudaError_t launch_el_output(const Op<T>& op, int batch, const double* u, T* strain, T* stress,
                             double* partials, double* results, SolverScalars* sc, cudaStream_t st) {
  k_el_output<T><<<post_grid_b((long long)op.nx * op.ny, batch), kPostThreads, 0, st>>>(
      op, u, strain, stress, partials, results, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_diff_stats(const Op<T>& op, int batch, const double* phi, double hdiff,
                              double c_macro, double* partials, double* results, SolverScalars* sc,
                              cudaStream_t st) {
  k_diff_stats<T><<<post_grid_b((long long)op.nx * op.ny, batch), kPostThreads, 0, st>>>(
      op, phi, hdiff, c_macro, partials, results, sc);
  return cudaGetLastError();
}
cudaError_t launch_diff_write_c(int nx, int ny, int batch, const uint8_t* phase, const double* phi,
                                double hdiff, double G0, double G1, const double* Gp, const double* beta_dev,
                                double* c, cudaStream_t st) {
  const long long total = (long long)nx * ny * batch;
  k_diff_write_c<<<post_grid(total), kPostThreads, 0, st>>>(nx, ny, total, phase, phi, hdiff, G0, G1, Gp,
                                                            beta_dev, c);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_history(long long N, int batch, const uint8_t* phase, double lam0, double lam1,
                           double mu0, double mu1, const T* strain, const T* eig, T* H, double* Hd,
                           double a, double* m0b, double* partials, SolverScalars* sc,
                           cudaStream_t st) {
  k_history<T><<<post_grid_b(N, batch), kPostThreads, 0, st>>>(N, phase, lam0, lam1, mu0, mu1, strain,
                                                               eig, H, Hd, a, m0b, partials, sc);
  return cudaGetLastError();
}
cudaError_t launch_pf_stats(long long N, int batch, const uint8_t* phase, const double* d,
                            double* partials, double* results, SolverScalars* sc, double Dp,
                            double Ds, double ih2, double* m1b, cudaStream_t st) {
  k_pf_stats<<<post_grid_b(N, batch), kPostThreads, 0, st>>>(N, phase, d, partials, results, sc, Dp, Ds,
                                                            ih2, m1b);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_degradation(long long N, const double* d, double kappa, T* g, cudaStream_t st) {
  k_degradation<T><<<post_grid(N), kPostThreads, 0, st>>>(N, d, kappa, g);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_precipitate(long long N, const uint8_t* phase, const double* c, double S,
                               double M, T* c_ppt, T* eig, cudaStream_t st) {
  k_precipitate<T><<<post_grid(N), kPostThreads, 0, st>>>(N, phase, c, S, M, c_ppt, eig);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale_copy(long long N, const T* src, double scale, T* dst, cudaStream_t st) {
  k_scale_copy<T><<<post_grid(N), kPostThreads, 0, st>>>(N, src, scale, dst);
  return cudaGetLastError();
}
cudaError_t launch_set_masked(long long N, const uint8_t* mask, double value, double* c,
                              cudaStream_t st) {
  k_set_masked<<<post_grid(N), kPostThreads, 0, st>>>(N, mask, value, c);
  return cudaGetLastError();
}
cudaError_t launch_df_split(long long n, const double* u, float* uh, float* ul, cudaStream_t st) {
  k_df_split<<<post_grid(n), kPostThreads, 0, st>>>(n, u, uh, ul);
  return cudaGetLastError();
}
cudaError_t launch_df_merge(long long n, const float* uh, const float* ul, double* u, cudaStream_t st) {
  k_df_merge<<<post_grid(n), kPostThreads, 0, st>>>(n, uh, ul, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_to_real(long long N, const double* src, T* dst, cudaStream_t st) {
  k_to_real<T><<<post_grid(N), kPostThreads, 0, st>>>(N, src, dst);
  return cudaGetLastError();
}

#define FFTMECH_POST_INST(T)                                                                       \
  template cudaError_t launch_el_output<T>(const Op<T>&, int, const double*, T*, T*, double*,     \
                                           double*, SolverScalars*, cudaStream_t);                 \
  template cudaError_t launch_diff_stats<T>(const Op<T>&, int, const double*, double, double,     \
                                            double*, double*, SolverScalars*, cudaStream_t);       \
  template cudaError_t launch_history<T>(long long, int, const uint8_t*, double, double, double,   \
                                         double, const T*, const T*, T*, double*, double, double*, \
                                         double*, SolverScalars*, cudaStream_t);                   \
  template cudaError_t launch_degradation<T>(long long, const double*, double, T*, cudaStream_t);  \
  template cudaError_t launch_precipitate<T>(long long, const uint8_t*, const double*, double,     \
                                             double, T*, T*, cudaStream_t);                        \
  template cudaError_t launch_scale_copy<T>(long long, const T*, double, T*, cudaStream_t);        \
  template cudaError_t launch_to_real<T>(long long, const double*, T*, cudaStream_t);

FFTMECH_POST_INST(float)
FFTMECH_POST_INST(double)

// Finalise a deferred column pass that no direction kernel followed (the
// solve stopped at its iteration limit): one block per problem.
template <typename T>
static __global__ void __launch_bounds__(256) k_col_finalize(const double* pcol, int ncol, SolverScalars* sc,
                                                             double invN) {
  __shared__ float redf[64];
  __shared__ double red[32];
  sc += blockIdx.x;
  if (done_flag(sc)) return;
  const double tot = deferred_total<T>(pcol + (size_t)blockIdx.x * ncol, ncol, redf, red);
  if (threadIdx.x == 0) finalize_col(sc, vol_readi(&sc->col_true) ? COL_TRUE : COL_ITER, tot * invN);
}

cudaError_t launch_col_finalize(const double* pcol, int ncol, SolverScalars* sc, int batch, double invN, int fp32,
                                cudaStream_t st) {
  if (fp32) k_col_finalize<float><<<batch, 256, 0, st>>>(pcol, ncol, sc, invN);
  else k_col_finalize<double><<<batch, 256, 0, st>>>(pcol, ncol, sc, invN);
  return cudaGetLastError();
}

}  // namespace fftmech
