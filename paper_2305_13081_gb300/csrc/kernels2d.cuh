// 2D row and column kernels that are not part of the split iteration: the
// FP64 true residual (r = b - K u, then the x transform into the packed
// spectrum), the column pass of every iteration (column FFT, multiplier
// 1 / (m0 + m1 |D|^2), Parseval <r, M^-1 r>, inverse FFT; two real
// components packed as one complex field, exact because the multiplier is
// real and even) and the bare row transform. Equivalence with the paper's
// projected gradient-space CG: G = D (D^-1) of App. A (Eq. g-42) maps
// potential PCG iterates onto gradient CG iterates one to one.
#pragma once

#include <atomic>

#include <algorithm>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"
#include "fftc.cuh"

namespace fftmech {

// Threads per block are capped at 512 (128 registers per thread available).
#define FFTMECH_BOUNDS(T) __launch_bounds__(512)

// ---------------------------------------------------------------- residual
// r = b - K u in the residual's number type (FP64 path: double; mixed path:
// double-float, ResidNum) with u from the iterate (zero_u: u = 0 except
// Dirichlet voxels), written as T and row-transformed into S. Shared memory:
// [max(D (R+2) numbers, 2 R T) per column] + [3 (R+1) numbers per column]
// (a number is 8 bytes either way).
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS(T) k_residual(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R, int zero_u,
                                             int filter) {
  using RN = typename ResidNum<T>::type;
  static_assert(sizeof(RN) == sizeof(double), "the shared-memory layout assumes 8-byte numbers");
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  grid_dep_sync();  // the plan is constant; everything below follows the previous kernel
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  if (filter == 1 && !(v.mode && v.mode[bp] != 0)) return;  // only problems being replaced / restarted
  if (filter == 2 && !unchecked_stop(v.sc + bp)) return;       // only newly stopped problems
  problem_views<T, D>(op, v, bp, N);
  const int y0 = blockIdx.x * R;
  const int rows = min(R, ny - y0);
  const int W = rows + 2;
  const size_t reg0 = (size_t)max(D * (R + 2) * (int)sizeof(RN), 2 * R * (int)sizeof(T)) * nx;
  RN* P = reinterpret_cast<RN*>(smem);
  RN* SG = reinterpret_cast<RN*>(smem + ((reg0 + 15) & ~size_t(15)));
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  const int SR = (rows + 1) * nx;  // stride of one SG component
  const RN zero = rn_f<RN>(0.f), one = rn_f<RN>(1.f);
  const RN ih = rn_c<RN>(1.0 / op.h);
  const RN E0 = rn_c<RN>(op.E[0]), E1 = rn_c<RN>(op.E[1]), E2 = rn_c<RN>(op.E[2]);
  const RN LAM[2] = {rn_c<RN>(op.lam[0]), rn_c<RN>(op.lam[1])};
  const RN MU[2] = {rn_c<RN>(op.mu[0]), rn_c<RN>(op.mu[1])};
  const RN KAP[2] = {rn_c<RN>(op.kap[0]), rn_c<RN>(op.kap[1])};
  const RN G0 = rn_c<RN>(D == 1 ? macro_grad(op, bp, 0) : 0.0), G1 = rn_c<RN>(D == 1 ? macro_grad(op, bp, 1) : 0.0);

  for (int i = threadIdx.x; i < W * nx; i += blockDim.x) {
    const int yy = i / nx, x = i - yy * nx;
    const size_t gi = (size_t)wrap_y(y0 - 1 + yy, ny) * nx + x;
    const bool keep = (D == 1) && op.mask && op.mask[gi];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      RN val;
      if constexpr (sizeof(T) == 4) val = RN{v.uh[c * N + gi], v.ul[c * N + gi]};
      else val = v.u[c * N + gi];
      if (zero_u && !keep) val = zero;
      P[(size_t)c * W * nx + i] = val;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SR; i += blockDim.x) {
    const int yy = i / nx, x = i - yy * nx;
    const int xp = (x + 1 == nx) ? 0 : x + 1;
    const size_t gi = (size_t)wrap_y(y0 - 1 + yy, ny) * nx + x;
    const int ph = op.phase[gi] ? 1 : 0;
    if constexpr (D == 2) {
      const RN* Ux = P;
      const RN* Uy = P + (size_t)W * nx;
      const int c0 = yy * nx + x;
      RN exx = (Ux[yy * nx + xp] - Ux[c0]) * ih + E0;
      RN eyy = (Uy[c0 + nx] - Uy[c0]) * ih + E1;
      const RN exy = (((Ux[c0 + nx] - Ux[c0]) + (Uy[yy * nx + xp] - Uy[c0])) * ih) * 0.5f + E2;
      const RN e = op.eig ? rn_t<RN>(op.eig[gi]) : zero;
      exx = exx - e;
      eyy = eyy - e;
      const RN gg = op.g ? rn_t<RN>(op.g[gi]) : one;
      const RN lam = gg * LAM[ph], mu = gg * MU[ph];
      const RN tr = exx + eyy;
      RN t0 = zero, t1 = zero, t2 = zero;  // prescribed stress (Voigt xx, yy, xy)
      if (op.pre) {
        t0 = rn_t<RN>(op.pre[gi]);
        t1 = rn_t<RN>(op.pre[N + gi]);
        t2 = rn_t<RN>(op.pre[2 * N + gi]);
      }
      SG[i] = lam * tr + (mu * exx) * 2.0f - t0;
      SG[SR + i] = lam * tr + (mu * eyy) * 2.0f - t1;
      SG[2 * SR + i] = (mu * exy) * 2.0f - t2;
    } else {
      const int c0 = yy * nx + x;
      const RN u = P[c0];
      const RN kap = KAP[ph];
      SG[i] = kap * ((P[yy * nx + xp] - u) * ih + G0);
      SG[SR + i] = kap * ((P[c0 + nx] - u) * ih + G1);
      SG[2 * SR + i] = u;
    }
  }
  __syncthreads();
  const RN C0C = rn_c<RN>(op.c0c), SRCS = rn_c<RN>(op.src_scale);
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) {
    const int yr = i / nx, x = i - yr * nx;
    const int yy = yr + 1;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const size_t gi = (size_t)(y0 + yr) * nx + x;
    const int c = yy * nx + x;
    RN r0, r1 = zero;
    if constexpr (D == 2) {
      const RN* Sxx = SG;
      const RN* Syy = SG + SR;
      const RN* Sxy = SG + 2 * SR;
      r0 = -(((Sxx[yy * nx + xm] - Sxx[c]) + (Sxy[c - nx] - Sxy[c])) * ih);
      r1 = -(((Sxy[yy * nx + xm] - Sxy[c]) + (Syy[c - nx] - Syy[c])) * ih);
    } else {
      const RN* Jx = SG;
      const RN* Jy = SG + SR;
      const RN div = ((Jx[yy * nx + xm] - Jx[c]) + (Jy[c - nx] - Jy[c])) * ih;
      const RN u = SG[2 * SR + c];
      const RN c0 = C0C + (op.c0f ? rn_t<RN>(op.c0f[gi]) : zero);
      const RN src = op.srcd ? rn_c<RN>(op.srcd[gi]) : (op.srct ? rn_t<RN>(op.srct[gi]) : zero);
      r0 = SRCS * src - c0 * u - div;
      if (op.mask && op.mask[gi]) r0 = zero;
    }
    const T t0 = (T)rn_out(r0), t1 = (T)rn_out(r1);
    v.r[gi] = t0;
    if constexpr (D == 2) v.r[N + gi] = t1;
    F[i] = mk(t0, t1);
  }
  __syncthreads();
  fft_lines<T, -1, FX>(F, px_s, rows, nx, 1, false);
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) v.S[(size_t)y0 * nx + i] = F[i];
}

// ---------------------------------------------------------------- column pass
// Column transform of a strip: the compile-time plan (NY > 0, CWC columns,
// blocks of col_threads<CWC>() threads) or the runtime one (nc columns).
constexpr int kColThreads = 512;
template <int CWC>
__host__ __device__ constexpr int col_threads() { return CWC >= 4 ? kColThreads : 256; }
template <typename T, int S, int FY, int NY, int CWC>
__device__ __forceinline__ void col_fft(cx<T>* B, const FftPlanDev<T>& p, int nc) {
  if constexpr (NY > 0) fftc<T, S, NY, true, CWC, col_threads<CWC>()>(B, p.tw, CWC);
  else fft_lines<T, S, FY>(B, p, nc, 1, nc, true);
}

// Multiplier of the column pass applied to one spectral value (frequency ky
// of strip column c): m = 1 / (m0 + m1 (lamx[c] + lamy[ky])), sum m |w|^2
// (Parseval), w <- w m / N unless the pass only measures the norm.
template <typename T>
struct ColMul {
  const T* lx;
  const T* ly;
  T m0, m1, invN;
  bool store;
  T part;
  int cnt;
  Acc<T>* acc;
  __device__ __forceinline__ void operator()(cx<T>& w, int ky, int c) {
    const T den = m0 + m1 * (lx[c] + ly[ky]);
    T m;
    if constexpr (sizeof(T) == 4) m = den > T(0) ? __fdividef(1.0f, den) : T(0);
    else m = den > T(0) ? T(1) / den : T(0);
    part += m * (w.re * w.re + w.im * w.im);
    if (++cnt == 16) {  // non-negative terms
      acc->add(part);
      part = T(0);
      cnt = 0;
    }
    if (store) w = scal(w, m * invN);
  }
};

// Strip of up to CW columns of S (stored [ky][c] in shared memory). Forward
// column FFT, multiply by m(k) / N, accumulate sum m |S|^2 (Parseval:
// <r, M^-1 r> = (1/N) sum_k m(k) |S(k)|^2 for the packed field), inverse
// column FFT. COL_PLAIN: one column FFT only (sign from `inverse`).
// One strip of the column pass (see k_colpass).
template <typename T, int FY, int NY, int CWC>
__device__ __forceinline__ void colpass_strip(int strip, int nx, int ny, cx<T>* S, cx<T>* B, const FftPlanDev<T>& py_s,
                                              const Spec<T>& sp, const T* lamx_s, const T* lamy_s, int CW, int mode,
                                              int inverse, int bp, Acc<T>& acc) {
  // with a compile-time plan the block size and the column length are
  // constants: the strip loops' row and column indices fold into offsets
  const int bd = NY > 0 ? col_threads<CWC>() : (int)blockDim.x;
  if constexpr (NY > 0) ny = NY;
  const int x0 = strip * CW;
  const int nc = min(CW, nx - x0);
  // shared rows: ncs columns; a compile-time plan always transforms CWC
  // columns (those past nc are zero and never stored or summed)
  const int ncs = NY > 0 ? CWC : nc;
  const int n = ny * ncs;
  const FastDiv dc(ncs);
  // staged strip load, 8 loads in flight per thread
  for (int i = threadIdx.x; i < n; i += 8 * bd) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * bd;
      if (ii < n) {
        const int y = NY > 0 ? ii / (CWC > 0 ? CWC : 1) : dc.div(ii), c = ii - y * ncs;
        t[k] = c < nc ? S[(size_t)y * nx + x0 + c] : mk(T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * bd < n) B[i + k * bd] = t[k];
  }
  __syncthreads();
  const bool store = (mode != COL_NORM && mode != COL_TRUENORM);
  if (mode == COL_PLAIN) {
    if (inverse) col_fft<T, 1, FY, NY, CWC>(B, py_s, ncs);
    else col_fft<T, -1, FY, NY, CWC>(B, py_s, ncs);
  } else if constexpr (NY > 0) {
    // compile-time plan: the multiplier and the Parseval sum are applied to
    // the last forward pass's outputs before they are stored
    const T m0 = sp.m0b ? (T)sp.m0b[bp] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[bp] : sp.m1_t;
    ColMul<T> mul{lamx_s, lamy_s, m0, m1, sp.invN_t, store, T(0), 0, &acc};
    fftc<T, -1, NY, true, CWC, col_threads<CWC>()>(B, py_s.tw, CWC, mul);
    acc.add(mul.part);
    if (store) {
      __syncthreads();
      col_fft<T, 1, FY, NY, CWC>(B, py_s, ncs);
    }
  } else {
    col_fft<T, -1, FY, NY, CWC>(B, py_s, ncs);
  }
  if (mode != COL_PLAIN && NY == 0) {
    const T m0 = sp.m0b ? (T)sp.m0b[bp] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[bp] : sp.m1_t;
    const T invN = sp.invN_t;
    T part = T(0);
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += bd) {
      const int ky = dc.div(i), c = i - ky * ncs;
      if (c >= nc) continue;
      const T den = m0 + m1 * (lamx_s[c] + lamy_s[ky]);
      T m;
      if constexpr (sizeof(T) == 4) m = den > T(0) ? __fdividef(1.0f, den) : T(0);
      else m = den > T(0) ? T(1) / den : T(0);
      const cx<T> w = B[i];
      part += m * (w.re * w.re + w.im * w.im);
      if (++cnt == 16) { acc.add(part); part = T(0); cnt = 0; }  // non-negative terms
      if (store) B[i] = scal(w, m * invN);
    }
    acc.add(part);
    if (store) {
      __syncthreads();
      col_fft<T, 1, FY, NY, CWC>(B, py_s, ncs);
    }
  }
  if (store) {
    for (int i = threadIdx.x; i < n; i += bd) {
      const int y = NY > 0 ? i / (CWC > 0 ? CWC : 1) : dc.div(i), c = i - y * ncs;
      if (c < nc) S[(size_t)y * nx + x0 + c] = B[i];
    }
  }
}

template <typename T, int FY, int NY, int CWC>
__global__ void FFTMECH_BOUNDS(T) k_colpass(int nx, int ny, cx<T>* S, FftPlanDev<T> py, Spec<T> sp, int CW,
                                            int mode_arg, int inverse, double* partials, SolverScalars* sc,
                                            int* pmode) {
  int mode = mode_arg & ~COL_DEFER;
  const int bp = blockIdx.y;
  S += (size_t)bp * nx * ny;
  if (sc) sc += bp;
  if (partials) partials += (size_t)bp * gridDim.x;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(py.n);
  const FftPlanDev<T> py_s = plan_to_smem(py, reinterpret_cast<cx<T>*>(smem_all));
  // the strip's symbol tables (constant) behind the strip buffer
  T* LY = reinterpret_cast<T*>(smem + (size_t)ny * CW * sizeof(cx<T>));
  T* LX = LY + ny;
  if (sp.lamy) {
    for (int i = threadIdx.x; i < ny; i += blockDim.x) LY[i] = sp.lamy[i];
    const int x0 = blockIdx.x * CW;
    if (threadIdx.x < CW) LX[threadIdx.x] = x0 + (int)threadIdx.x < nx ? sp.lamx[x0 + threadIdx.x] : T(0);
  }
  grid_dep_sync();  // plan and tables are constant; everything below follows the previous kernel
  if (mode == COL_ITER && pmode && pmode[bp] == 1) mode = COL_TRUE;  // reliable update of this problem
  if (mode == COL_RESTART && !(pmode && pmode[bp] == 2)) return;      // only restarting problems
  if (mode == COL_TRUENORM && sc && !unchecked_stop(sc)) return;      // only newly stopped problems
  if (mode != COL_PLAIN && mode != COL_NORM && mode != COL_TRUENORM && mode != COL_RESTART &&
      done_flag(sc))
    return;
  __shared__ double red[32];
  __shared__ float redf[64];
  cx<T>* B = reinterpret_cast<cx<T>*>(smem);
  // one strip per block (a loop over strips around the transform costs the
  // compiler about twice the registers)
  Acc<T> acc;
  colpass_strip<T, FY, NY, CWC>(blockIdx.x, nx, ny, S, B, py_s, sp, LX, LY, CW, mode, inverse, bp, acc);
  if (mode == COL_PLAIN) return;
  // every mode stores its partial in the deferred format, so a total formed
  // here (last block) and one formed by the next direction kernel agree bit
  // for bit
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

// Plain row FFT of S (used by the stand-alone transform).
template <typename T, int FX>
__global__ void FFTMECH_BOUNDS(T) k_rowfft(int nx, int ny, cx<T>* S, FftPlanDev<T> px, int R, int inverse) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  const int y0 = blockIdx.x * R;
  const int rows = min(R, ny - y0);
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) F[i] = S[(size_t)y0 * nx + i];
  __syncthreads();
  if (inverse) fft_lines<T, 1, FX>(F, px_s, rows, nx, 1, false);
  else fft_lines<T, -1, FX>(F, px_s, rows, nx, 1, false);
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) S[(size_t)y0 * nx + i] = F[i];
}

// ---------------------------------------------------------------- launchers

template <typename T, int D, int FX>
cudaError_t launch_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                            const Shape2& sh, int zero_u, int filter, cudaStream_t st) {
  const int R = sh.rows_res;
  const size_t sm = smem_residual<T, D>(op.nx, R) + tw_smem_bytes<T>(op.nx);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_residual<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((op.ny + R - 1) / R, sh.batch);
  return launch_dep(k_residual<T, D, FX>, grid, dim3(sh.threads_res), sm, st, op, v, px, R, zero_u, filter);
}

template <typename T, int FY, int NY, int CWC>
cudaError_t launch_colpass(int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp,
                           const Shape2& sh, int mode, int inverse, double* partials,
                           SolverScalars* sc, int* pmode, cudaStream_t st) {
  const int CW = sh.cols;
  const size_t sm = (size_t)ny * CW * sizeof(cx<T>) + tw_smem_bytes<T>(ny) + (size_t)(ny + CW) * sizeof(T);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_colpass<T, FY, NY, CWC>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((nx + CW - 1) / CW, sh.batch > 0 ? sh.batch : 1);
  return launch_dep(k_colpass<T, FY, NY, CWC>, grid, dim3(NY > 0 ? col_threads<CWC>() : sh.threads_col), sm, st, nx, ny,
                    S, py, sp, CW, mode, inverse, partials, sc, pmode);
}

template <typename T, int FX>
cudaError_t launch_rowfft(int nx, int ny, cx<T>* S, const FftPlanDev<T>& px, int inverse,
                          const Shape2& sh, cudaStream_t st) {
  const int R = sh.rows_update;
  const size_t sm = (size_t)R * nx * sizeof(cx<T>) + tw_smem_bytes<T>(nx);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_rowfft<T, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const int grid = (ny + R - 1) / R;
  k_rowfft<T, FX><<<grid, sh.threads_update, sm, st>>>(nx, ny, S, px, R, inverse);
  return cudaGetLastError();
}

// Explicit instantiations for one radix family (one translation unit each).
#define FFTMECH_INST_TD(T, D, F)                                                                   \
  template cudaError_t launch_residual<T, D, F>(const Op<T>&, const Vec2<T>&,                    \
                                                const FftPlanDev<T>&, const Shape2&, int, int,    \
                                                cudaStream_t);
#define FFTMECH_INST_T(T, F)                                                                       \
  FFTMECH_INST_TD(T, 1, F)                                                                         \
  FFTMECH_INST_TD(T, 2, F)                                                                         \
  template cudaError_t launch_colpass<T, F, 0, 0>(int, int, cx<T>*, const FftPlanDev<T>&,         \
                                            const Spec<T>&, const Shape2&, int, int, double*,    \
                                            SolverScalars*, int*, cudaStream_t);            \
  template cudaError_t launch_rowfft<T, F>(int, int, cx<T>*, const FftPlanDev<T>&, int,           \
                                           const Shape2&, cudaStream_t);
// column passes of a compile-time length (float) for strips of 4 or 8 columns
#define FFTMECH_INST_COL_FIXED(NY)                                                                               \
  template cudaError_t launch_colpass<float, FAM_ALL, NY, 2>(int, int, cx<float>*, const FftPlanDev<float>&,    \
                                                             const Spec<float>&, const Shape2&, int, int,       \
                                                             double*, SolverScalars*, int*, cudaStream_t); \
  template cudaError_t launch_colpass<float, FAM_ALL, NY, 4>(int, int, cx<float>*, const FftPlanDev<float>&,    \
                                                             const Spec<float>&, const Shape2&, int, int,       \
                                                             double*, SolverScalars*, int*, cudaStream_t); \
  template cudaError_t launch_colpass<float, FAM_ALL, NY, 8>(int, int, cx<float>*, const FftPlanDev<float>&,    \
                                                             const Spec<float>&, const Shape2&, int, int,       \
                                                             double*, SolverScalars*, int*, cudaStream_t);
#define FFTMECH_INST_FAMILY(F) \
  FFTMECH_INST_T(float, F)     \
  FFTMECH_INST_T(double, F)

}  // namespace fftmech
