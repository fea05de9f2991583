// FP64 post-processing of the 3D solves: strain / stress output with volume
// averages, diffusion statistics and concentration, history field. The
// pointwise kernels that do not look at neighbours (precipitation,
// degradation, phase-field statistics) are shared with 2D.
#include "fftmech_internal.cuh"
#include "fftmech.h"

namespace fftmech {

static constexpr int kPost3Threads = 256;

static inline dim3 post3_grid(long long n, int batch) {
  long long g = (n + kPost3Threads - 1) / kPost3Threads;
  const long long cap = batch > 1 ? 512 : 4096;
  if (g > cap) g = cap;
  return dim3((unsigned)(g < 1 ? 1 : g), (unsigned)batch);
}

// Voxel gi of an [nz][ny][nx] grid and its forward neighbours (periodic).
struct Nbr3 {
  int x, y, z;
  long long ixp, iyp, izp;
  __device__ Nbr3(long long gi, int nx, int ny, int nz) {
    const long long plane = (long long)nx * ny;
    z = (int)(gi / plane);
    const long long rem = gi - (long long)z * plane;
    y = (int)(rem / nx);
    x = (int)(rem - (long long)y * nx);
    const long long base = gi - x;
    ixp = base + (x + 1 == nx ? 0 : x + 1);
    iyp = (long long)z * plane + (long long)(y + 1 == ny ? 0 : y + 1) * nx + x;
    izp = (long long)(z + 1 == nz ? 0 : z + 1) * plane + (long long)y * nx + x;
  }
};

// strain = E + sym grad+ u (Voigt xx, yy, zz, yz, xz, xy; tensor shear),
// stress = g C : (strain - e I) (Eq. solid); per problem sums of stress,
// strain and the energy density 1/2 (strain - e I) : stress ->
// results[b * 13 + k].
template <typename T>
__global__ void k3_el_output(Op<T> op, const double* __restrict__ u, T* strain, T* stress, double* partials,
                             double* results, SolverScalars* sc) {
  __shared__ double red[32 * 13];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long long N = (long long)nx * ny * nz;
  const int b = blockIdx.y;
  const size_t o1 = (size_t)b * N;
  u += 3 * o1;
  if (strain) strain += 6 * o1;
  if (stress) stress += 6 * o1;
  const uint8_t* phase = op.phase + o1;
  const T* g = op.g ? op.g + o1 : nullptr;
  const T* eig = op.eig ? op.eig + o1 : nullptr;
  partials += (size_t)b * gridDim.x * 13;
  const double ih = 1.0 / op.h;
  double acc[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double* ux = u;
  const double* uy = u + N;
  const double* uz = u + 2 * N;
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const Nbr3 q(gi, nx, ny, nz);
    double e[6];
    e[0] = op.E[0] + (ux[q.ixp] - ux[gi]) * ih;
    e[1] = op.E[1] + (uy[q.iyp] - uy[gi]) * ih;
    e[2] = op.E[2] + (uz[q.izp] - uz[gi]) * ih;
    e[3] = op.E[3] + 0.5 * ((uy[q.izp] - uy[gi]) + (uz[q.iyp] - uz[gi])) * ih;
    e[4] = op.E[4] + 0.5 * ((ux[q.izp] - ux[gi]) + (uz[q.ixp] - uz[gi])) * ih;
    e[5] = op.E[5] + 0.5 * ((ux[q.iyp] - ux[gi]) + (uy[q.ixp] - uy[gi])) * ih;
    const double ev = eig ? (double)eig[gi] : 0.0;
    const int ph = phase[gi] ? 1 : 0;
    const double gg = g ? (double)g[gi] : 1.0;
    const double lam = gg * op.lam[ph], mu = gg * op.mu[ph];
    double a[6] = {e[0] - ev, e[1] - ev, e[2] - ev, e[3], e[4], e[5]};
    const double lt = lam * (a[0] + a[1] + a[2]);
    double s[6];
    for (int k = 0; k < 3; ++k) s[k] = lt + 2 * mu * a[k];
    for (int k = 3; k < 6; ++k) s[k] = 2 * mu * a[k];
    for (int k = 0; k < 6; ++k) {
      if (strain) strain[k * N + gi] = (T)e[k];
      if (stress) stress[k * N + gi] = (T)s[k];
      acc[k] += s[k];
      acc[6 + k] += e[k];
    }
    acc[12] += 0.5 * (a[0] * s[0] + a[1] * s[1] + a[2] * s[2] + 2 * (a[3] * s[3] + a[4] * s[4] + a[5] * s[5]));
  }
  block_sum<13>(acc, red);
  if (publish_partials<13>(acc, partials, &sc[b].cnt[2])) {
    double tot[13];
    gather_partials<13>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0)
      for (int k = 0; k < 13; ++k) results[b * 13 + k] = tot[k];
  }
}

// Phase statistics of the homogenised diffusion solution (Eq. psi-two-values)
// and the mean flux; results[b * 7 + .]: beta_pore, beta_solid, <jx>, <jy>,
// <jz>, porosity, c_macro of the problem.
template <typename T>
__global__ void k3_diff_stats(Op<T> op, const double* __restrict__ phi, double hdiff, double c_macro,
                              double* partials, double* results, SolverScalars* sc) {
  __shared__ double red[32 * 9];
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const long long N = (long long)nx * ny * nz;
  const int b = blockIdx.y;
  phi += (size_t)b * N;
  const uint8_t* phase = op.phase + (size_t)b * N;
  partials += (size_t)b * gridDim.x * 9;
  const double ih = 1.0 / hdiff;
  const double G0 = macro_grad(op, b, 0), G1 = macro_grad(op, b, 1), G2 = macro_grad(op, b, 2);
  if (op.cmp) c_macro = op.cmp[b];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < N;
       gi += (long long)gridDim.x * blockDim.x) {
    const Nbr3 q(gi, nx, ny, nz);
    const int s = phase[gi] ? 1 : 0;  // 0 pore, 1 solid
    const double ramp = G0 * (q.x * hdiff) + G1 * (q.y * hdiff) + G2 * (q.z * hdiff);
    acc[s] += 1.0;
    acc[2 + s] += phi[gi];
    acc[4 + s] += ramp;
    const double D = op.kap[s];
    acc[6] += -D * (G0 + (phi[q.ixp] - phi[gi]) * ih);
    acc[7] += -D * (G1 + (phi[q.iyp] - phi[gi]) * ih);
    acc[8] += -D * (G2 + (phi[q.izp] - phi[gi]) * ih);
  }
  block_sum<9>(acc, red);
  if (publish_partials<9>(acc, partials, &sc[b].cnt[2])) {
    double tot[9];
    gather_partials<9>(tot, partials, &sc[b].cnt[2], red);
    if (threadIdx.x == 0) {
      const double np = tot[0], ns = tot[1];
      const double eta = np / (double)N;
      double* r = results + b * 7;
      r[0] = np > 0 ? c_macro / eta - (tot[4] + tot[2]) / np : 0.0;
      r[1] = ns > 0 ? -(tot[5] + tot[3]) / ns : 0.0;
      r[2] = tot[6] / (double)N;
      r[3] = tot[7] / (double)N;
      r[4] = tot[8] / (double)N;
      r[5] = eta;
      r[6] = c_macro;
    }
  }
}

// c = grad c_mac . x + phi + beta_phase (Eqs. concentration,
// concentration-correct), beta of problem b from results[b * 7 + 0 / 1];
// Gp: per-problem gradients (NULL: G0, G1, G2 for all).
__global__ void k3_diff_write_c(int nx, int ny, int nz, long long total, const uint8_t* __restrict__ phase,
                                const double* __restrict__ phi, double hdiff, double G0, double G1, double G2,
                                const double* __restrict__ Gp, const double* __restrict__ beta,
                                double* __restrict__ c) {
  const long long N = (long long)nx * ny * nz;
  for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < total;
       gi += (long long)gridDim.x * blockDim.x) {
    const long long b = gi / N, li = gi - b * N;
    const Nbr3 q(li, nx, ny, nz);
    const double bt = phase[gi] ? beta[b * 7 + 1] : beta[b * 7 + 0];
    const double* g = Gp ? Gp + 3 * b : nullptr;
    const double g0 = g ? g[0] : G0, g1 = g ? g[1] : G1, g2 = g ? g[2] : G2;
    c[gi] = g0 * (q.x * hdiff) + g1 * (q.y * hdiff) + g2 * (q.z * hdiff) + phi[gi] + bt;
  }
}

// H = max(H, psi+(eps - e I)) with Eq. (energy) in d = 3 (bulk factor
// lambda + 2 mu / 3, deviator eps - tr(eps)/3 I); Hd = H as double; per
// problem m0b[b] = a + mean(H).
template <typename T>
__global__ void k3_history(long long N, const uint8_t* __restrict__ phase, double lam0, double lam1, double mu0,
                           double mu1, const T* __restrict__ strain, const T* __restrict__ eig, T* H, double* Hd,
                           double a, double* m0b, double* partials, SolverScalars* sc) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const size_t o1 = (size_t)b * N;
  phase += o1;
  strain += 6 * o1;
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
    const double exx = (double)strain[gi] - e, eyy = (double)strain[N + gi] - e, ezz = (double)strain[2 * N + gi] - e;
    const double eyz = (double)strain[3 * N + gi], exz = (double)strain[4 * N + gi], exy = (double)strain[5 * N + gi];
    const double tr = exx + eyy + ezz;
    const double dx = exx - tr / 3.0, dy = eyy - tr / 3.0, dz = ezz - tr / 3.0;
    const double trp = tr > 0 ? tr : 0.0;
    const double K = lam + 2.0 * mu / 3.0;
    const double psi =
        0.5 * K * trp * trp + mu * (dx * dx + dy * dy + dz * dz + 2 * (exy * exy + exz * exz + eyz * eyz));
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

// ---------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch3_el_output(const Op<T>& op, int batch, const double* u, T* strain, T* stress, double* partials,
                              double* results, SolverScalars* sc, cudaStream_t st) {
  k3_el_output<T><<<post3_grid((long long)op.nx * op.ny * op.nz, batch), kPost3Threads, 0, st>>>(
      op, u, strain, stress, partials, results, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch3_diff_stats(const Op<T>& op, int batch, const double* phi, double hdiff, double c_macro,
                               double* partials, double* results, SolverScalars* sc, cudaStream_t st) {
  k3_diff_stats<T><<<post3_grid((long long)op.nx * op.ny * op.nz, batch), kPost3Threads, 0, st>>>(
      op, phi, hdiff, c_macro, partials, results, sc);
  return cudaGetLastError();
}
cudaError_t launch3_diff_write_c(int nx, int ny, int nz, int batch, const uint8_t* phase, const double* phi,
                                 double hdiff, const double G[3], const double* Gp, const double* beta_dev,
                                 double* c, cudaStream_t st) {
  const long long total = (long long)nx * ny * nz * batch;
  long long g = (total + kPost3Threads - 1) / kPost3Threads;
  if (g > 4096) g = 4096;
  k3_diff_write_c<<<(unsigned)(g < 1 ? 1 : g), kPost3Threads, 0, st>>>(nx, ny, nz, total, phase, phi, hdiff, G[0],
                                                                       G[1], G[2], Gp, beta_dev, c);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch3_history(long long N, int batch, const uint8_t* phase, double lam0, double lam1, double mu0,
                            double mu1, const T* strain, const T* eig, T* H, double* Hd, double a, double* m0b,
                            double* partials, SolverScalars* sc, cudaStream_t st) {
  k3_history<T><<<post3_grid(N, batch), kPost3Threads, 0, st>>>(N, phase, lam0, lam1, mu0, mu1, strain, eig, H, Hd,
                                                                a, m0b, partials, sc);
  return cudaGetLastError();
}

#define FFTMECH_POST3_INST(T)                                                                                    \
  template cudaError_t launch3_el_output<T>(const Op<T>&, int, const double*, T*, T*, double*, double*,          \
                                            SolverScalars*, cudaStream_t);                                       \
  template cudaError_t launch3_diff_stats<T>(const Op<T>&, int, const double*, double, double, double*, double*, \
                                             SolverScalars*, cudaStream_t);                                      \
  template cudaError_t launch3_history<T>(long long, int, const uint8_t*, double, double, double, double,        \
                                          const T*, const T*, T*, double*, double, double*, double*,             \
                                          SolverScalars*, cudaStream_t);

FFTMECH_POST3_INST(float)
FFTMECH_POST3_INST(double)

}  // namespace fftmech
