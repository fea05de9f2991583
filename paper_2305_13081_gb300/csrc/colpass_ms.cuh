// Column pass of the 2D equilibrium PCG with the reference-medium
// preconditioner (the Moulinec-Suquet reference medium, Sec. 1): z = K0^-1 r
// per Fourier mode, K0 the Galerkin operator grad+^T C0 grad+ of a
// homogeneous isotropic medium (lambda0 = rho mu0, mu0 = 1). With
// a = D h (forward-difference symbol, Sec. 2.6) the mode matrix is
//   K0(k) = |a|^2 I + rho conj(a) a^T + a conj(a)^T        (Hermitian 2 x 2)
// and z(k) = h^2 / m1 K0(k)^-1 r(k) (0 at k = 0), the same scale as the
// Laplace preconditioner 1 / (m1 |D|^2).
//
// The two displacement components travel packed, S = F(r_x + i r_y), so a
// mode's components need the value at -k as well:
//   R_x(k) = (S(k) + conj(S(-k))) / 2,  R_y(k) = (S(k) - conj(S(-k))) / (2 i),
// and the result is packed back as S'(k) = z_x(k) + i z_y(k),
// S'(-k) = conj(z_x(k)) + i conj(z_y(k)) (real fields: z(-k) = conj(z(k))).
// A block therefore holds a strip of CW columns kx in [0, nx / 2] and their
// mirror columns nx - kx: y-FFT of both, the 2 x 2 solve of every mode pair
// (one thread per pair), the Parseval sum <r, M^-1 r> (each pair counted for
// both of its modes), the inverse y-FFT and the stores. Columns kx = 0 and
// kx = nx / 2 are their own mirrors; their pairs are (ky, -ky) inside the
// column. Partials, deferred totals and the last-block finalisation follow
// the Laplace column pass exactly.
// NY > 0: compile-time plan of NY points (float, CW = 4, 512 threads);
// NY = 0: the runtime plan of family FY.
#pragma once

#include "kernels2d.cuh"

namespace fftmech {

template <typename T, int FY, int NY>
__global__ void FFTMECH_BOUNDS(T) k_colpass_ms(int nx, int ny, cx<T>* S, FftPlanDev<T> py, Spec<T> sp, int CW,
                                               int mode_arg, double* partials, SolverScalars* sc, int* pmode) {
  int mode = mode_arg & ~COL_DEFER;
  const int bp = blockIdx.y;
  S += (size_t)bp * nx * ny;
  sc += bp;
  partials += (size_t)bp * gridDim.x;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(py.n);
  const FftPlanDev<T> py_s = plan_to_smem(py, reinterpret_cast<cx<T>*>(smem_all));
  const int ncs = NY > 0 ? 8 : 2 * CW;  // lower columns in slots 0 .. CW - 1, mirrors in CW .. 2 CW - 1
  const int bd = NY > 0 ? kColThreads : (int)blockDim.x;  // a constant with a compile-time plan
  if constexpr (NY > 0) ny = NY;
  cx<T>* B = reinterpret_cast<cx<T>*>(smem);
  cx<T>* AY = B + (size_t)ny * ncs;
  cx<T>* AX = AY + ny;
  const int H = nx / 2 + 1;
  const int x0 = blockIdx.x * CW;
  const int nc = min(CW, H - x0);
  for (int i = threadIdx.x; i < ny; i += bd) AY[i] = sp.ay[i];
  if ((int)threadIdx.x < CW) AX[threadIdx.x] = (int)threadIdx.x < nc ? sp.ax[x0 + threadIdx.x] : mk(T(0), T(0));
  grid_dep_sync();  // plan and tables are constant; everything below follows the previous kernel
  if (mode == COL_ITER && pmode && pmode[bp] == 1) mode = COL_TRUE;  // reliable update of this problem
  if (mode == COL_RESTART && !(pmode && pmode[bp] == 2)) return;      // only restarting problems
  if (mode == COL_TRUENORM && !unchecked_stop(sc)) return;            // only newly stopped problems
  if (mode != COL_NORM && mode != COL_TRUENORM && mode != COL_RESTART && done_flag(sc)) return;
  __shared__ double red[32];
  __shared__ float redf[64];
  const int n = ny * ncs;
  const FastDiv dn(ncs);
  for (int i = threadIdx.x; i < n; i += 8 * bd) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * bd;
      if (ii < n) {
        const int y = NY > 0 ? ii / 8 : dn.div(ii), s = ii - y * ncs;
        const int c = s < CW ? s : s - CW;
        const int kx = x0 + c;
        const int col = s < CW ? kx : (kx == 0 ? 0 : nx - kx);
        t[k] = c < nc ? S[(size_t)y * nx + col] : mk(T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * bd < n) B[i + k * bd] = t[k];
  }
  __syncthreads();
  if constexpr (NY > 0) fftc<T, -1, NY, true, 8, kColThreads>(B, py_s.tw, 8);  // CW = 4: 8 columns
  else fft_lines<T, -1, FY>(B, py_s, ncs, 1, ncs, true);
  __syncthreads();
  const bool store = (mode != COL_NORM && mode != COL_TRUENORM);
  const T m1 = sp.m1b ? (T)sp.m1b[bp] : sp.m1_t;
  const T invN = sp.invN_t;
  const T rho = sp.rho_t;
  Acc<T> acc;
  T part = T(0);
  int cnt = 0;
  const FastDiv dc(nc);
  for (int i = threadIdx.x; i < ny * nc; i += bd) {
    const int ky = dc.div(i), c = i - ky * nc;
    const int kx = x0 + c;
    const bool self = kx == 0 || 2 * kx == nx;
    const int kyn = ky == 0 ? 0 : ny - ky;
    if (self && ky > kyn) continue;  // the pair belongs to row kyn
    const int ia = ky * ncs + c;
    const int ib = self ? kyn * ncs + c : kyn * ncs + CW + c;
    const cx<T> a = B[ia], b = B[ib];
    const cx<T> Rx = mk(T(0.5) * (a.re + b.re), T(0.5) * (a.im - b.im));
    const cx<T> Ry = mk(T(0.5) * (a.im + b.im), T(-0.5) * (a.re - b.re));
    const cx<T> ax = AX[c], ay = AY[ky];
    const T lx = ax.re * ax.re + ax.im * ax.im, ly = ay.re * ay.re + ay.im * ay.im;
    const T s2 = lx + ly;
    cx<T> zx = mk(T(0), T(0)), zy = mk(T(0), T(0));
    if (s2 > T(0)) {
      // w = conj(a_x) a_y; K12 = rho w + conj(w)
      const T wre = ax.re * ay.re + ax.im * ay.im, wim = ax.re * ay.im - ax.im * ay.re;
      const T k12r = (rho + T(1)) * wre, k12i = (rho - T(1)) * wim;
      const T k11 = s2 + (rho + T(1)) * lx, k22 = s2 + (rho + T(1)) * ly;
      const T det = k11 * k22 - (k12r * k12r + k12i * k12i);
      T f;
      if constexpr (sizeof(T) == 4) f = __fdividef(1.0f, m1 * det);
      else f = T(1) / (m1 * det);
      // z = f [[k22, -K12], [-conj(K12), k11]] R
      zx = mk(f * (k22 * Rx.re - (k12r * Ry.re - k12i * Ry.im)), f * (k22 * Rx.im - (k12r * Ry.im + k12i * Ry.re)));
      zy = mk(f * (k11 * Ry.re - (k12r * Rx.re + k12i * Rx.im)), f * (k11 * Ry.im - (k12r * Rx.im - k12i * Rx.re)));
    }
    const T w2 = (self && ky == kyn) ? T(1) : T(2);
    part += w2 * (Rx.re * zx.re + Rx.im * zx.im + Ry.re * zy.re + Ry.im * zy.im);
    if (++cnt == 16) {  // non-negative terms
      acc.add(part);
      part = T(0);
      cnt = 0;
    }
    if (store) {
      zx = scal(zx, invN);
      zy = scal(zy, invN);
      B[ia] = mk(zx.re - zy.im, zx.im + zy.re);
      if (ib != ia) B[ib] = mk(zx.re + zy.im, zy.re - zx.im);
    }
  }
  acc.add(part);
  if (store) {
    __syncthreads();
    if constexpr (NY > 0) fftc<T, 1, NY, true, 8, kColThreads>(B, py_s.tw, 8);
    else fft_lines<T, 1, FY>(B, py_s, ncs, 1, ncs, true);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += bd) {
      const int y = NY > 0 ? i / 8 : dn.div(i), s = i - y * ncs;
      const int c = s < CW ? s : s - CW;
      const int kx = x0 + c;
      if (c >= nc) continue;
      if (s < CW) S[(size_t)y * nx + kx] = B[i];
      else if (!(kx == 0 || 2 * kx == nx)) S[(size_t)y * nx + (nx - kx)] = B[i];
    }
  }
  store_deferred_partial<T>(acc, partials + blockIdx.x, redf, red);
  if ((mode_arg & COL_DEFER) && (mode == COL_ITER || mode == COL_TRUE)) {  // finalised by the next direction kernel
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->col_true = mode == COL_TRUE;
    return;
  }
  __shared__ int am_last;
  if (threadIdx.x == 0) am_last = ticket_acq_rel(&sc->cnt[1]) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  const double tot = deferred_total<T>(partials, gridDim.x, redf, red);
  if (threadIdx.x == 0) {
    sc->cnt[1] = 0u;
    finalize_col(sc, mode, tot * sp.invN, pmode ? pmode + bp : nullptr);
  }
}

template <typename T, int FY, int NY>
cudaError_t launch_colpass_ms(int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp, int CW,
                              int threads, int batch, int mode, double* partials, SolverScalars* sc, int* pmode,
                              cudaStream_t st) {
  const size_t sm = (size_t)ny * 2 * CW * sizeof(cx<T>) + (size_t)(ny + CW) * sizeof(cx<T>) + tw_smem_bytes<T>(ny);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_colpass_ms<T, FY, NY>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(colpass_ms_blocks(nx, CW), batch > 0 ? batch : 1);
  return launch_dep(k_colpass_ms<T, FY, NY>, grid, dim3(NY > 0 ? kColThreads : threads), sm, st, nx, ny, S, py, sp, CW, mode, partials, sc,
                    pmode);
}

#define FFTMECH_MS_SIG(T)                                                                                   \
  (int, int, cx<T>*, const FftPlanDev<T>&, const Spec<T>&, int, int, int, int, double*, SolverScalars*, int*, \
   cudaStream_t)
// Explicit instantiation of the compile-time-plan variant for length N.
#define FFTMECH_INST_COL_MS_FIXED(N) \
  template cudaError_t launch_colpass_ms<float, FAM_ALL, N> FFTMECH_MS_SIG(float);

}  // namespace fftmech
