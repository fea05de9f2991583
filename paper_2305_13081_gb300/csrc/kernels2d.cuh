// 2D kernels of the FFT-Galerkin preconditioned CG (potential form).
//
// One PCG iteration is three launches on the row-major grid [ny][nx]:
//   direction (rows): z = row-IFFT(S); p = z + beta p_old; <p, K p> (energy form)
//   update    (rows): u += alpha p; r -= alpha K p; S = row-FFT(r packed re/im)
//   column    (strips of columns): S = col-IFFT(m(k) col-FFT(S)); <r, M^-1 r>
// where M^-1 = F^-1 diag(m) F is the Fourier multiplier 1 / (m0 + m1 |D|^2)
// applied per component (two real components packed as one complex field,
// exact because m is real and even). Equivalence with the paper's projected
// gradient-space CG: G = D (D^-1) of App. A (Eq. g-42) maps potential PCG
// iterates onto gradient CG iterates one to one.
#pragma once

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

// Threads per block are capped at 512 (128 registers per thread available).
#define FFTMECH_BOUNDS(T) __launch_bounds__(512)

// ---------------------------------------------------------------- residual
// r = b - K u in FP64 (u from the iterate, zero_u: u = 0 except Dirichlet
// voxels), written as T and row-transformed into S. Shared memory:
// [max(D (R+2) doubles, 2 R T) per column] + [3 (R+1) doubles per column].
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS(T) k_residual(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R, int zero_u,
                                             int filter) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  if (filter && !(v.mode && v.mode[bp] != 0)) return;  // only problems being replaced / restarted
  problem_views<T, D>(op, v, bp, N);
  const int y0 = blockIdx.x * R;
  const int rows = min(R, ny - y0);
  const int W = rows + 2;
  const size_t reg0 = (size_t)max(D * (R + 2) * (int)sizeof(double), 2 * R * (int)sizeof(T)) * nx;
  double* P = reinterpret_cast<double*>(smem);
  double* SG = reinterpret_cast<double*>(smem + ((reg0 + 15) & ~size_t(15)));
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  const int SR = (rows + 1) * nx;  // stride of one SG component
  const double ih = 1.0 / op.h;

  for (int i = threadIdx.x; i < W * nx; i += blockDim.x) {
    const int yy = i / nx, x = i - yy * nx;
    const size_t gi = (size_t)wrap_y(y0 - 1 + yy, ny) * nx + x;
    const bool keep = (D == 1) && op.mask && op.mask[gi];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double val;
      if constexpr (sizeof(T) == 4) val = (double)v.uh[c * N + gi] + (double)v.ul[c * N + gi];
      else val = v.u[c * N + gi];
      if (zero_u && !keep) val = 0.0;
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
      const double* Ux = P;
      const double* Uy = P + (size_t)W * nx;
      const int c0 = yy * nx + x;
      double exx = (Ux[yy * nx + xp] - Ux[c0]) * ih + op.E[0];
      double eyy = (Uy[c0 + nx] - Uy[c0]) * ih + op.E[1];
      const double exy = 0.5 * ((Ux[c0 + nx] - Ux[c0]) + (Uy[yy * nx + xp] - Uy[c0])) * ih + op.E[2];
      const double e = op.eig ? (double)op.eig[gi] : 0.0;
      exx -= e;
      eyy -= e;
      const double gg = op.g ? (double)op.g[gi] : 1.0;
      const double lam = gg * op.lam[ph], mu = gg * op.mu[ph];
      const double tr = exx + eyy;
      SG[i] = lam * tr + 2.0 * mu * exx;
      SG[SR + i] = lam * tr + 2.0 * mu * eyy;
      SG[2 * SR + i] = 2.0 * mu * exy;
    } else {
      const int c0 = yy * nx + x;
      const double u = P[c0];
      const double kap = op.kap[ph];
      SG[i] = kap * ((P[yy * nx + xp] - u) * ih + op.G[0]);
      SG[SR + i] = kap * ((P[c0 + nx] - u) * ih + op.G[1]);
      SG[2 * SR + i] = u;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) {
    const int yr = i / nx, x = i - yr * nx;
    const int yy = yr + 1;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const size_t gi = (size_t)(y0 + yr) * nx + x;
    const int c = yy * nx + x;
    double r0, r1 = 0.0;
    if constexpr (D == 2) {
      const double* Sxx = SG;
      const double* Syy = SG + SR;
      const double* Sxy = SG + 2 * SR;
      r0 = -((Sxx[yy * nx + xm] - Sxx[c]) + (Sxy[c - nx] - Sxy[c])) * ih;
      r1 = -((Sxy[yy * nx + xm] - Sxy[c]) + (Syy[c - nx] - Syy[c])) * ih;
    } else {
      const double* Jx = SG;
      const double* Jy = SG + SR;
      const double div = ((Jx[yy * nx + xm] - Jx[c]) + (Jy[c - nx] - Jy[c])) * ih;
      const double u = SG[2 * SR + c];
      const double c0 = op.c0c + (op.c0f ? (double)op.c0f[gi] : 0.0);
      const double src = op.srcd ? op.srcd[gi] : (op.srct ? (double)op.srct[gi] : 0.0);
      r0 = op.src_scale * src - c0 * u - div;
      if (op.mask && op.mask[gi]) r0 = 0.0;
    }
    const T t0 = (T)r0, t1 = (T)r1;
    v.r[gi] = t0;
    if constexpr (D == 2) v.r[N + gi] = t1;
    F[i] = mk(t0, t1);
  }
  __syncthreads();
  fft_lines<T, -1, FX>(F, px_s, rows, nx, 1, false);
  for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) v.S[(size_t)y0 * nx + i] = F[i];
}

// ---------------------------------------------------------------- update
// u += alpha p (FP64 iterate); r -= alpha K p; S = row-FFT(r). Every input
// of the tile (direction rows with halos, old residual, phase, degradation or
// reaction field, mask) is staged into shared memory first with many loads in
// flight; the stencil then runs out of shared memory (layout UpdLayout).
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS(T) k_update(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R) {
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  const int u_only = v.mode ? (v.mode[bp] == 1) : 0;  // reliable update: iterate only
  problem_views<T, D>(op, v, bp, N);
  if (done_flag(v.sc)) return;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  // alpha: a double for the FP64 path, a float pair (ah + al) for MIXED
  double alpha = 0.0;
  float ah = 0.f, al = 0.f;
  if constexpr (sizeof(T) == 4) {
    ah = vol_readf(&v.sc->alpha_h);
    al = vol_readf(&v.sc->alpha_l);
  } else {
    alpha = vol_read(&v.sc->alpha);
  }
  const T a = sizeof(T) == 4 ? (T)ah : (T)alpha;
  const int y0 = blockIdx.x * R;
  const int rows = min(R, ny - y0);
  const int tid = threadIdx.x, bd = blockDim.x;
  const size_t t0 = (size_t)y0 * nx;
  if (u_only) {
    // reliable-update iteration: only the iterate moves (direction from global)
    for (int c = 0; c < D; ++c) {
      const T* p = v.p_in + c * N + t0;
      if constexpr (sizeof(T) == 4) {
        float* uh = v.uh + c * N + t0;
        float* ul = v.ul + c * N + t0;
        for (int i = tid; i < rows * nx; i += bd) {
          float h = uh[i], l = ul[i];
          df_axpy(h, l, ah, al, (float)p[i]);
          uh[i] = h;
          ul[i] = l;
        }
      } else {
        double* u = v.u + c * N + t0;
        for (int i = tid; i < rows * nx; i += bd) u[i] += alpha * (double)p[i];
      }
    }
    return;
  }
  const UpdLayout L(nx, R, (int)sizeof(T), D);
  T* P = reinterpret_cast<T*>(smem + L.a);
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + L.a);
  T* SG = reinterpret_cast<T*>(smem + L.b);
  T* RS = reinterpret_cast<T*>(smem + L.c);
  T* MG = reinterpret_cast<T*>(smem + L.d);
  uint8_t* PH = smem + L.e;
  uint8_t* MK = smem + L.f;
  const int W = rows + 2;
  const int SR = (rows + 1) * nx;
  const T* matg = (D == 2) ? op.g : op.c0f;
  // stage the tile
#pragma unroll
  for (int c = 0; c < D; ++c) g2s_rows<8>(P + (size_t)c * W * nx, v.p_in + c * N, y0 - 1, W, nx, ny);
#pragma unroll
  for (int c = 0; c < D; ++c) g2s_vec<8, false>(RS + (size_t)c * rows * nx, v.r + c * N + t0, rows * nx);
  if (matg) g2s_rows<8>(MG, matg, y0 - 1, rows + 1, nx, ny);
  g2s_rows<8>(PH, op.phase, y0 - 1, rows + 1, nx, ny);
  const bool masked = (D == 1) && op.mask;
  if (masked) g2s_vec<8, true>(MK, op.mask + t0, rows * nx);
  __syncthreads();
  // iterate update on the tile rows (rows 1 .. rows of P)
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < D; ++c)
      df_axpy_g<8>(v.uh + c * N + t0, v.ul + c * N + t0, P + (size_t)c * W * nx + nx, ah, al, rows * nx);
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) axpy_g<8>(v.u + c * N + t0, P + (size_t)c * W * nx + nx, alpha, rows * nx);
  }
  // stresses (D = 2) or fluxes (D = 1) at rows y0 - 1 .. y0 + rows - 1
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  for (int yy = 0; yy <= rows; ++yy) {
    for (int x = tid; x < nx; x += bd) {
      const int xp = (x + 1 == nx) ? 0 : x + 1;
      const int i = yy * nx + x;
      const bool sol = PH[i] != 0;
      if constexpr (D == 2) {
        const T* Ux = P;
        const T* Uy = P + (size_t)W * nx;
        const T exx = (Ux[yy * nx + xp] - Ux[i]) * ih;
        const T eyy = (Uy[i + nx] - Uy[i]) * ih;
        const T exy = T(0.5) * ((Ux[i + nx] - Ux[i]) + (Uy[yy * nx + xp] - Uy[i])) * ih;
        const T gg = matg ? MG[i] : T(1);
        const T lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
        const T tr = exx + eyy;
        SG[i] = lam * tr + T(2) * mu * exx;
        SG[SR + i] = lam * tr + T(2) * mu * eyy;
        SG[2 * SR + i] = T(2) * mu * exy;
      } else {
        const T p = P[i];
        const T kap = sol ? kap1 : kap0;
        SG[i] = kap * (P[yy * nx + xp] - p) * ih;
        SG[SR + i] = kap * (P[i + nx] - p) * ih;
        SG[2 * SR + i] = (c0c + (matg ? MG[i] : T(0))) * p;
      }
    }
  }
  __syncthreads();
  // K p, residual update and packing (F reuses the direction rows)
  for (int yr = 0; yr < rows; ++yr) {
    for (int x = tid; x < nx; x += bd) {
      const int yy = yr + 1;
      const int xm = (x == 0) ? nx - 1 : x - 1;
      const int c = yy * nx + x;
      const int j = yr * nx + x;
      T r0, r1 = T(0);
      if constexpr (D == 2) {
        const T* Sxx = SG;
        const T* Syy = SG + SR;
        const T* Sxy = SG + 2 * SR;
        const T q0 = ((Sxx[yy * nx + xm] - Sxx[c]) + (Sxy[c - nx] - Sxy[c])) * ih;
        const T q1 = ((Sxy[yy * nx + xm] - Sxy[c]) + (Syy[c - nx] - Syy[c])) * ih;
        r0 = RS[j] - a * q0;
        r1 = RS[rows * nx + j] - a * q1;
        v.r[t0 + j] = r0;
        v.r[N + t0 + j] = r1;
      } else {
        const T* Jx = SG;
        const T* Jy = SG + SR;
        T q0 = SG[2 * SR + c] + ((Jx[yy * nx + xm] - Jx[c]) + (Jy[c - nx] - Jy[c])) * ih;
        if (masked && MK[j]) q0 = T(0);
        r0 = RS[j] - a * q0;
        v.r[t0 + j] = r0;
      }
      F[j] = mk(r0, r1);
    }
  }
  __syncthreads();
  fft_lines<T, -1, FX>(F, px_s, rows, nx, 1, false);
  s2g(v.S + t0, F, rows * nx);
}

// ---------------------------------------------------------------- direction
// z = row-IFFT(S) (rows y0 .. y0 + rows, one halo row), p = z + beta p_old,
// <p, K p> = sum of the energy density over the tile (layout DirLayout).
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS(T) k_direction(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R) {
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  problem_views<T, D>(op, v, bp, N);
  if (done_flag(v.sc)) return;
  double* partials = v.partials + (size_t)bp * gridDim.x;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  __shared__ double red[32];
  __shared__ float redf[64];
  T b;
  if constexpr (sizeof(T) == 4) b = vol_readf(&v.sc->beta_f);
  else b = vol_read(&v.sc->beta);
  const int y0 = blockIdx.x * R;
  const int rows = min(R, ny - y0);
  const int W = rows + 1;
  const int tid = threadIdx.x, bd = blockDim.x;
  const size_t t0 = (size_t)y0 * nx;
  const DirLayout L(nx, R, (int)sizeof(T), D);
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + L.a);
  T* P = reinterpret_cast<T*>(smem + L.b);
  T* MG = reinterpret_cast<T*>(smem + L.c);
  uint8_t* PH = smem + L.d;
  uint8_t* MK = smem + L.e;
  const T* matg = (D == 2) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  g2s_rows<8>(F, v.S, y0, W, nx, ny);
  const bool with_old = b != T(0);  // the first iteration has p = z
  if (with_old) {
#pragma unroll
    for (int c = 0; c < D; ++c) g2s_rows<8>(P + (size_t)c * W * nx, v.p_in + c * N, y0, W, nx, ny);
  }
  if (matg) g2s_vec<8, true>(MG, matg + t0, rows * nx);
  g2s_vec<8, true>(PH, op.phase + t0, rows * nx);
  if (masked) g2s_rows<8>(MK, op.mask, y0, W, nx, ny);
  __syncthreads();
  fft_lines<T, 1, FX>(F, px_s, W, nx, 1, false);
  for (int yy = 0; yy < W; ++yy) {
    for (int x = tid; x < nx; x += bd) {
      const int i = yy * nx + x;
      const cx<T> z = F[i];
      T p0 = z.re;
      if (masked && MK[i]) p0 = T(0);
      if (with_old) p0 += b * P[i];
      P[i] = p0;
      if (yy < rows) v.p_out[t0 + i] = p0;
      if constexpr (D == 2) {
        T p1 = z.im;
        if (with_old) p1 += b * P[(size_t)W * nx + i];
        P[(size_t)W * nx + i] = p1;
        if (yy < rows) v.p_out[N + t0 + i] = p1;
      }
    }
  }
  __syncthreads();
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  Acc<T> acc;
  for (int yy = 0; yy < rows; ++yy) {
    T part = T(0);
    for (int x = tid; x < nx; x += bd) {
      const int xp = (x + 1 == nx) ? 0 : x + 1;
      const int i = yy * nx + x;
      const bool sol = PH[i] != 0;
      T w;
      if constexpr (D == 2) {
        const T* Ux = P;
        const T* Uy = P + (size_t)W * nx;
        const T exx = (Ux[yy * nx + xp] - Ux[i]) * ih;
        const T eyy = (Uy[i + nx] - Uy[i]) * ih;
        const T exy = T(0.5) * ((Ux[i + nx] - Ux[i]) + (Uy[yy * nx + xp] - Uy[i])) * ih;
        const T gg = matg ? MG[i] : T(1);
        const T lam = sol ? lam1 : lam0, mu = sol ? mu1 : mu0;
        const T tr = exx + eyy;
        w = gg * (lam * tr * tr + T(2) * mu * (exx * exx + eyy * eyy + T(2) * exy * exy));
      } else {
        const T p = P[i];
        const T gx = (P[yy * nx + xp] - p) * ih, gy = (P[i + nx] - p) * ih;
        const T c0v = c0c + (matg ? MG[i] : T(0));
        w = c0v * p * p + (sol ? kap1 : kap0) * (gx * gx + gy * gy);
      }
      part += w;  // a few terms per thread and row, all non-negative
    }
    acc.add(part);
  }
  const double bt[1] = {acc.block_total(redf, red)};
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- column pass
// Strip of up to CW columns of S (stored [ky][c] in shared memory). Forward
// column FFT, multiply by m(k) / N, accumulate sum m |S|^2 (Parseval:
// <r, M^-1 r> = (1/N) sum_k m(k) |S(k)|^2 for the packed field), inverse
// column FFT. COL_PLAIN: one column FFT only (sign from `inverse`).
template <typename T, int FY>
__global__ void FFTMECH_BOUNDS(T) k_colpass(int nx, int ny, cx<T>* S, FftPlanDev<T> py, Spec<T> sp, int CW,
                                            int mode, int inverse, double* partials, SolverScalars* sc,
                                            const int* pmode) {
  const int bp = blockIdx.y;
  S += (size_t)bp * nx * ny;
  if (sc) sc += bp;
  if (partials) partials += (size_t)bp * gridDim.x;
  if (mode == COL_ITER && pmode && pmode[bp] == 1) mode = COL_TRUE;  // reliable update of this problem
  if (mode == COL_RESTART && !(pmode && pmode[bp] == 2)) return;      // only restarting problems
  if (mode != COL_PLAIN && mode != COL_NORM && mode != COL_TRUENORM && mode != COL_RESTART &&
      done_flag(sc))
    return;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(py.n);
  const FftPlanDev<T> py_s = plan_to_smem(py, reinterpret_cast<cx<T>*>(smem_all));
  __shared__ double red[32];
  __shared__ float redf[64];
  cx<T>* B = reinterpret_cast<cx<T>*>(smem);
  const int x0 = blockIdx.x * CW;
  const int nc = min(CW, nx - x0);
  const int n = ny * nc;
  const int bd = blockDim.x;
  const FastDiv dc(nc);
  // staged strip load, 8 loads in flight per thread
  for (int i = threadIdx.x; i < n; i += 8 * bd) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * bd;
      if (ii < n) {
        const int y = dc.div(ii), c = ii - y * nc;
        t[k] = S[(size_t)y * nx + x0 + c];
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * bd < n) B[i + k * bd] = t[k];
  }
  __syncthreads();
  if (mode == COL_PLAIN) {
    if (inverse) fft_lines<T, 1, FY>(B, py_s, nc, 1, nc, true);
    else fft_lines<T, -1, FY>(B, py_s, nc, 1, nc, true);
  } else {
    fft_lines<T, -1, FY>(B, py_s, nc, 1, nc, true);
  }
  const bool store = (mode != COL_NORM && mode != COL_TRUENORM);
  Acc<T> acc;
  if (mode != COL_PLAIN) {
    const T m0 = sp.m0b ? (T)sp.m0b[bp] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[bp] : sp.m1_t;
    const T invN = sp.invN_t;
    T part = T(0);
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += bd) {
      const int ky = dc.div(i), c = i - ky * nc;
      const T den = m0 + m1 * (sp.lamx[x0 + c] + sp.lamy[ky]);
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
      fft_lines<T, 1, FY>(B, py_s, nc, 1, nc, true);
    }
  }
  if (store) {
    for (int i = threadIdx.x; i < n; i += bd) {
      const int y = dc.div(i), c = i - y * nc;
      S[(size_t)y * nx + x0 + c] = B[i];
    }
  }
  if (mode == COL_PLAIN) return;
  const double bt[1] = {acc.block_total(redf, red)};
  if (publish_partials<1>(bt, partials, &sc->cnt[1])) {
    double tot[1];
    gather_partials<1>(tot, partials, &sc->cnt[1], red);
    if (threadIdx.x == 0) finalize_col(sc, mode, tot[0] * sp.invN);
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
// Opt every row / column kernel into the device's full dynamic shared memory
// once per process (launches then pass their own, smaller, sizes).
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes, int& configured) {
  if (configured) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in limit
  if ((long long)bytes > (long long)dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e == cudaSuccess) configured = 1;
  return e;
}

template <typename T, int D, int FX>
cudaError_t launch_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                            const Shape2& sh, int zero_u, int filter, cudaStream_t st) {
  const int R = sh.rows_res;
  const size_t sm = smem_residual<T, D>(op.nx, R) + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem(k_residual<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((op.ny + R - 1) / R, sh.batch);
  k_residual<T, D, FX><<<grid, sh.threads_res, sm, st>>>(op, v, px, R, zero_u, filter);
  return cudaGetLastError();
}

template <typename T, int D, int FX>
cudaError_t launch_update(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                          const Shape2& sh, cudaStream_t st) {
  const int R = sh.rows_update;
  const size_t sm = smem_update<T, D>(op.nx, R) + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem(k_update<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((op.ny + R - 1) / R, sh.batch);
  k_update<T, D, FX><<<grid, sh.threads_update, sm, st>>>(op, v, px, R);
  return cudaGetLastError();
}

template <typename T, int D, int FX>
cudaError_t launch_direction(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                             const Shape2& sh, cudaStream_t st) {
  const int R = sh.rows_dir;
  const size_t sm = smem_direction<T, D>(op.nx, R) + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem(k_direction<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((op.ny + R - 1) / R, sh.batch);
  k_direction<T, D, FX><<<grid, sh.threads_dir, sm, st>>>(op, v, px, R);
  return cudaGetLastError();
}

template <typename T, int FY>
cudaError_t launch_colpass(int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp,
                           const Shape2& sh, int mode, int inverse, double* partials,
                           SolverScalars* sc, const int* pmode, cudaStream_t st) {
  const int CW = sh.cols;
  const size_t sm = (size_t)ny * CW * sizeof(cx<T>) + tw_smem_bytes<T>(ny);
  static int cfg = 0;
  cudaError_t e = set_smem(k_colpass<T, FY>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((nx + CW - 1) / CW, sh.batch > 0 ? sh.batch : 1);
  k_colpass<T, FY><<<grid, sh.threads_col, sm, st>>>(nx, ny, S, py, sp, CW, mode, inverse, partials, sc,
                                                     pmode);
  return cudaGetLastError();
}

template <typename T, int FX>
cudaError_t launch_rowfft(int nx, int ny, cx<T>* S, const FftPlanDev<T>& px, int inverse,
                          const Shape2& sh, cudaStream_t st) {
  const int R = sh.rows_update;
  const size_t sm = (size_t)R * nx * sizeof(cx<T>) + tw_smem_bytes<T>(nx);
  static int cfg = 0;
  cudaError_t e = set_smem(k_rowfft<T, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const int grid = (ny + R - 1) / R;
  k_rowfft<T, FX><<<grid, sh.threads_update, sm, st>>>(nx, ny, S, px, R, inverse);
  return cudaGetLastError();
}

// Explicit instantiations for one radix family (one translation unit each).
#define FFTMECH_INST_TD(T, D, F)                                                                   \
  template cudaError_t launch_residual<T, D, F>(const Op<T>&, const Vec2<T>&,                    \
                                                const FftPlanDev<T>&, const Shape2&, int, int,    \
                                                cudaStream_t);                                    \
  template cudaError_t launch_update<T, D, F>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&, \
                                              const Shape2&, cudaStream_t);                       \
  template cudaError_t launch_direction<T, D, F>(const Op<T>&, const Vec2<T>&,                   \
                                                 const FftPlanDev<T>&, const Shape2&, cudaStream_t);
#define FFTMECH_INST_T(T, F)                                                                       \
  FFTMECH_INST_TD(T, 1, F)                                                                         \
  FFTMECH_INST_TD(T, 2, F)                                                                         \
  template cudaError_t launch_colpass<T, F>(int, int, cx<T>*, const FftPlanDev<T>&,               \
                                            const Spec<T>&, const Shape2&, int, int, double*,    \
                                            SolverScalars*, const int*, cudaStream_t);            \
  template cudaError_t launch_rowfft<T, F>(int, int, cx<T>*, const FftPlanDev<T>&, int,           \
                                           const Shape2&, cudaStream_t);
#define FFTMECH_INST_FAMILY(F) \
  FFTMECH_INST_T(float, F)     \
  FFTMECH_INST_T(double, F)

}  // namespace fftmech
