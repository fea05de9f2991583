// 3D kernels of the FFT-Galerkin preconditioned CG (potential form) on the
// grid [nz][ny][nx], x fastest, that are not x-line or stencil kernels: the
// FP64 true residual and the y / z line passes.
//
// The operator, multiplier and PCG recursion are those of 2D with a third
// direction: K u = grad+^T [g C : sym grad+ u] for the three displacement
// components (D = 3), or K u = c0 u + grad+^T [kap grad+ u] for a scalar
// (D = 1); the preconditioner is 1 / (m0 + m1 |D|^2) with |D|^2 = lam_x +
// lam_y + lam_z (the forward-difference symbol of Sec. 2.6 in the projection
// of App. A, Eq. g-42). An iteration runs the x-line and stencil kernels
// (lines.cuh, stencil.cuh) and then three line passes:
//   y pass (y lines): S = y-FFT(S)
//   z pass (z lines): S = z-IFFT(m(k) z-FFT(S)); <r, M^-1 r>
//   y pass (y lines): S = y-IFFT(S)
// Spectral rows: row (z, y) of S holds, for D = 3, the packed components
// (r_x + i r_y) as nx complex numbers followed by the half spectrum
// (nx/2 + 1 numbers) of r_z; for D = 1 only the half spectrum. A real line's
// spectrum is Hermitian, so the other half is never stored or transformed
// along y and z.
#pragma once

#include <atomic>

#include <algorithm>
#include <type_traits>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"
#include "fftc.cuh"

namespace fftmech {

#define FFTMECH_BOUNDS3 __launch_bounds__(512)

// Stress (D = 3) or flux (D = 1) components kept per plane: NP in-plane
// ones (differenced along x and y: sxx, syy, sxy or Jx, Jy) and NZ ones
// differenced along z (sxz, syz, szz or Jz), the latter in a two-plane ring.
// NF complex fields go through the x transform.
template <int D>
struct Comp3 {
  static constexpr int NP = D == 3 ? 3 : 2;
  static constexpr int NZ = D == 3 ? 3 : 1;
  static constexpr int NF = D == 3 ? 2 : 1;
};

template <typename T, int D>
__device__ __forceinline__ void problem_views3(Op<T>& op, Vec2<T>& v, int b, size_t N, long long sst) {
  const size_t o1 = (size_t)b * N, oD = (size_t)b * D * N;
  op.phase += o1;
  if (op.g) op.g += o1;
  if (op.eig) op.eig += o1;
  if (op.c0f) op.c0f += o1;
  if (op.mask) op.mask += o1;
  if (op.srcd) op.srcd += o1;
  if (op.srct) op.srct += o1;
  if (op.pre) op.pre += (size_t)b * (D == 3 ? 6 : 3) * N;
  if (v.u) v.u += oD;
  if (v.uh) v.uh += oD;
  if (v.ul) v.ul += oD;
  v.r += oD;
  if (v.p_in) v.p_in += oD;
  if (v.p_out) v.p_out += oD;
  v.S += (size_t)b * sst;
  v.sc += b;
}

static __device__ __forceinline__ int wrap_z(int z, int nz) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }

// FP64 iterate of plane z (periodic) into ring slot s of P: lines y0 - 1 ..
// y0 + W - 2 of every component (zero_u: 0 except on Dirichlet voxels).
template <typename T, int D, typename RN>
__device__ __forceinline__ void load_iterate3(RN* P, const Op<T>& op, const Vec2<T>& v, int z, int s, int y0,
                                              int W, size_t PS, size_t N, int zero_u) {
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const int zw = wrap_z(z, nz);
  RN* dst = P + (size_t)s * D * PS;
  const FastDiv dnx(nx);
  for (int i = threadIdx.x; i < W * nx; i += blockDim.x) {
    const int l = dnx.div(i), x = i - l * nx;
    const size_t gi = (size_t)zw * plane + (size_t)wrap_y(y0 - 1 + l, ny) * nx + x;
    const bool keep = (D == 1) && op.mask && op.mask[gi];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      RN val;
      if constexpr (sizeof(T) == 4) val = RN{v.uh[c * N + gi], v.ul[c * N + gi]};
      else val = v.u[c * N + gi];
      if (zero_u && !keep) val = rn_f<RN>(0.f);
      dst[c * PS + i] = val;
    }
  }
}

// ---------------------------------------------------------------- residual
// r = b - K u in the residual's number type (FP64 path: double; mixed path:
// double-float, ResidNum) from the iterate (zero_u: u = 0 except on
// Dirichlet voxels; filter: only problems with a nonzero mode), written as
// T; S = x-FFT(r). Bricks of R lines march through Zc planes keeping two
// planes of the iterate and of the z-differenced stress (or flux)
// components; plane zz = z0 - 1 is the halo (its z-differenced components
// only).
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS3 k3_residual(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R, int Zc, long long sst,
                                            int zero_u, int filter) {
  using C = Comp3<D>;
  using RN = typename ResidNum<T>::type;
  static_assert(sizeof(RN) == 8, "the shared-memory layout assumes 8-byte numbers");
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  grid_dep_sync();
  if (filter == 1 && !(v.mode && v.mode[bp] != 0)) return;  // only problems being replaced / restarted
  if (filter == 2 && !unchecked_stop(v.sc + bp)) return;       // only newly stopped problems
  problem_views3<T, D>(op, v, bp, N, sst);
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  const int nty = (ny + R - 1) / R;
  const int tz = blockIdx.x / nty, ty = blockIdx.x - tz * nty;
  const int y0 = ty * R, rows = min(R, ny - y0);
  const int z0 = tz * Zc, planes = min(Zc, nz - z0);
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nxa = D == 3 ? nx : 0, nxh = nx / 2 + 1, nxs = nxa + nxh;
  const Row3Layout L(nx, R, (int)sizeof(RN), (int)sizeof(T), D);
  RN* P = reinterpret_cast<RN*>(smem + L.P);
  RN* SP = reinterpret_cast<RN*>(smem + L.SP);
  RN* SZ = reinterpret_cast<RN*>(smem + L.SZ);
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + L.F);
  T* MG = reinterpret_cast<T*>(smem + L.MG);
  uint8_t* PH = smem + L.PH;
  const int W = rows + 2;                   // iterate lines y0 - 1 .. y0 + rows
  const size_t PS = (size_t)(R + 2) * nx;   // one component of one P slot
  const size_t SS = (size_t)(R + 1) * nx;   // one stress component of one plane
  const T* matg = (D == 3) ? op.g : op.c0f;
  const RN zero = rn_f<RN>(0.f), one = rn_f<RN>(1.f);
  const RN ih = rn_c<RN>(1.0 / op.h);
  RN E[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) E[k] = rn_c<RN>(D == 3 ? op.E[k] : macro_grad(op, bp, k < 3 ? k : 0));
  const RN LAM[2] = {rn_c<RN>(op.lam[0]), rn_c<RN>(op.lam[1])};
  const RN MU[2] = {rn_c<RN>(op.mu[0]), rn_c<RN>(op.mu[1])};
  const RN KAP[2] = {rn_c<RN>(op.kap[0]), rn_c<RN>(op.kap[1])};
  const RN C0C = rn_c<RN>(op.c0c), SRCS = rn_c<RN>(op.src_scale);
  const FastDiv dnx(nx);

  load_iterate3<T, D>(P, op, v, z0 - 1, 0, y0, W, PS, N, zero_u);
  for (int zz = z0 - 1; zz < z0 + planes; ++zz) {
    const int cur = (zz - z0 + 1) & 1, nxt = cur ^ 1;
    const bool inner = zz >= z0;
    const int zw = wrap_z(zz, nz);
    const size_t pz = (size_t)zw * plane;
    load_iterate3<T, D>(P, op, v, zz + 1, nxt, y0, W, PS, N, zero_u);
    if (matg) g2s_rows<4>(MG, matg + pz, y0 - 1, rows + 1, nx, ny);
    g2s_rows<4>(PH, op.phase + pz, y0 - 1, rows + 1, nx, ny);
    __syncthreads();
    const RN* Pc = P + (size_t)cur * D * PS;
    const RN* Pn = P + (size_t)nxt * D * PS;
    RN* Zc_ = SZ + (size_t)cur * C::NZ * SS;
    const RN* Zp = SZ + (size_t)nxt * C::NZ * SS;  // previous plane (same slot parity as the next)
    // stress / flux of plane zz at lines y0 - 1 .. y0 + rows - 1
    for (int i = tid; i < (rows + 1) * nx; i += bd) {
      const int l = dnx.div(i), x = i - l * nx;
      const int xp = (x + 1 == nx) ? 0 : x + 1;
      const int ix = l * nx + xp;
      const int ph = PH[i] != 0 ? 1 : 0;
      if constexpr (D == 3) {
        const RN* Ux = Pc;
        const RN* Uy = Pc + PS;
        const RN* Uz = Pc + 2 * PS;
        const RN ux = Ux[i], uy = Uy[i], uz = Uz[i];
        const size_t gi = pz + (size_t)wrap_y(y0 - 1 + l, ny) * nx + x;
        const RN e = op.eig ? rn_t<RN>(op.eig[gi]) : zero;
        const RN exx = (Ux[ix] - ux) * ih + E[0] - e;
        const RN eyy = (Uy[i + nx] - uy) * ih + E[1] - e;
        const RN ezz = (Pn[2 * PS + i] - uz) * ih + E[2] - e;
        const RN eyz = (((Pn[PS + i] - uy) + (Uz[i + nx] - uz)) * ih) * 0.5f + E[3];
        const RN exz = (((Pn[i] - ux) + (Uz[ix] - uz)) * ih) * 0.5f + E[4];
        const RN exy = (((Ux[i + nx] - ux) + (Uy[ix] - uy)) * ih) * 0.5f + E[5];
        const RN gg = matg ? rn_t<RN>(MG[i]) : one;
        const RN lam = gg * LAM[ph], mu = gg * MU[ph];
        const RN lt = lam * ((exx + eyy) + ezz);
        const RN m2 = mu * 2.0f;
        RN t[6] = {zero, zero, zero, zero, zero, zero};  // prescribed stress (Voigt xx, yy, zz, yz, xz, xy)
        if (op.pre) {
#pragma unroll
          for (int k = 0; k < 6; ++k) t[k] = rn_t<RN>(op.pre[k * N + gi]);
        }
        if (inner) {
          SP[i] = lt + m2 * exx - t[0];
          SP[SS + i] = lt + m2 * eyy - t[1];
          SP[2 * SS + i] = m2 * exy - t[5];
        }
        Zc_[i] = m2 * exz - t[4];
        Zc_[SS + i] = m2 * eyz - t[3];
        Zc_[2 * SS + i] = lt + m2 * ezz - t[2];
      } else {
        const RN p = Pc[i];
        const RN kap = KAP[ph];
        const RN gx = (Pc[ix] - p) * ih + E[0];
        const RN gy = (Pc[i + nx] - p) * ih + E[1];
        const RN gz = (Pn[i] - p) * ih + E[2];
        if (inner) {
          SP[i] = kap * gx;
          SP[SS + i] = kap * gy;
        }
        Zc_[i] = kap * gz;
      }
    }
    __syncthreads();
    if (!inner) continue;
    // residual on the interior lines, packed for the x transform
    for (int i = tid; i < rows * nx; i += bd) {
      const int lr = dnx.div(i), x = i - lr * nx;
      const int l = lr + 1;
      const int xm = (x == 0) ? nx - 1 : x - 1;
      const int c = l * nx + x, cxm = l * nx + xm;
      const size_t gi = pz + (size_t)(y0 + lr) * nx + x;
      if constexpr (D == 3) {
        const RN* Sxx = SP;
        const RN* Syy = SP + SS;
        const RN* Sxy = SP + 2 * SS;
        const RN* Sxz = Zc_;
        const RN* Syz = Zc_ + SS;
        const RN* Szz = Zc_ + 2 * SS;
        const T r0 = (T)rn_out(-((((Sxx[cxm] - Sxx[c]) + (Sxy[c - nx] - Sxy[c])) + (Zp[c] - Sxz[c])) * ih));
        const T r1 = (T)rn_out(-((((Sxy[cxm] - Sxy[c]) + (Syy[c - nx] - Syy[c])) + (Zp[SS + c] - Syz[c])) * ih));
        const T r2 = (T)rn_out(-((((Sxz[cxm] - Sxz[c]) + (Syz[c - nx] - Syz[c])) + (Zp[2 * SS + c] - Szz[c])) * ih));
        v.r[gi] = r0;
        v.r[N + gi] = r1;
        v.r[2 * N + gi] = r2;
        F[i] = mk(r0, r1);
        F[(size_t)rows * nx + i] = mk(r2, T(0));
      } else {
        const RN* Jx = SP;
        const RN* Jy = SP + SS;
        const RN div = (((Jx[cxm] - Jx[c]) + (Jy[c - nx] - Jy[c])) + (Zp[c] - Zc_[c])) * ih;
        const RN c0v = C0C + (matg ? rn_t<RN>(MG[c]) : zero);
        const RN src = op.srcd ? rn_c<RN>(op.srcd[gi]) : (op.srct ? rn_t<RN>(op.srct[gi]) : zero);
        RN rr = SRCS * src - c0v * Pc[c] - div;
        if (op.mask && op.mask[gi]) rr = zero;
        const T r0 = (T)rn_out(rr);
        v.r[gi] = r0;
        F[i] = mk(r0, T(0));
      }
    }
    __syncthreads();
    fft_lines_call<T, -1, FX>(F, px_s, C::NF * rows, nx, 1, false);
    // store: packed field in full, the real field's half spectrum
    cx<T>* Srow = v.S + ((size_t)zw * ny + y0) * nxs;
    const FastDiv dns(nxs);
    for (int i = tid; i < rows * nxs; i += bd) {
      const int l = dns.div(i), k = i - l * nxs;
      cx<T> w;
      if (k < nxa) w = F[(size_t)l * nx + k];
      else w = F[(size_t)(C::NF - 1) * rows * nx + (size_t)l * nx + (k - nxa)];
      Srow[i] = w;
    }
    __syncthreads();
  }
}

// Multiplier of the z pass applied to one spectral value (line frequency
// kl of strip column c): m = 1 / (m0 + m1 (lamc[c] + lamj + laml[kl])),
// Parseval sum wcol[c] m |w|^2, w <- w m / N unless only the norm is wanted.
template <typename T>
struct ZMul {
  const T* lc;
  const T* wc;
  const T* ll;
  T lj, m0, m1, invN;
  bool store;
  T part;
  int cnt;
  Acc<T>* acc;
  __device__ __forceinline__ void operator()(cx<T>& w, int kl, int c) {
    const T den = m0 + m1 * (lc[c] + lj + ll[kl]);
    T m;
    if constexpr (sizeof(T) == 4) m = den > T(0) ? __fdividef(1.0f, den) : T(0);
    else m = den > T(0) ? T(1) / den : T(0);
    part += wc[c] * m * (w.re * w.re + w.im * w.im);
    if (++cnt == 16) {  // non-negative terms
      acc->add(part);
      part = T(0);
      cnt = 0;
    }
    if (store) w = scal(w, m * invN);
  }
};

// ---------------------------------------------------------------- line passes
constexpr int kLineThreads = 512;  // block size of the compile-time-plan line passes
// A strip of CW spectral columns of one line set: nlines complex numbers per
// column, line_stride apart. Line set j of problem b starts at
// S + b sst + j set_stride (y pass: j = z plane; z pass: j = ky).
// stage 0 / 2: forward / inverse FFT along the lines (y pass).
// stage 1 (z pass): forward FFT, multiply by m(k) / N with
//   lambda = lamc[column] + lamj[j] + laml[line], sum of wcol m |S|^2
//   (Parseval over the full spectrum: the half-spectrum columns count
//   twice except kx = 0 and kx = nx/2), inverse FFT unless NORM/TRUENORM.
template <typename T, int FL, int NL, int CWC>
__global__ void FFTMECH_BOUNDS3 k3_lines(cx<T>* S, long long sst, int nset, long long set_stride, int nlines,
                                         long long line_stride, int ncols, FftPlanDev<T> pl, Spec<T> sp,
                                         int CW, int stage, int mode, double* partials, SolverScalars* sc,
                                         int* pmode) {
  const int b = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(pl.n);
  const FftPlanDev<T> pl_s = plan_to_smem(pl, reinterpret_cast<cx<T>*>(smem_all));
  // with a compile-time plan the block size and the line length are
  // constants: the strip loops' row and column indices fold into offsets
  const int bd = NL > 0 ? kLineThreads : (int)blockDim.x;
  if constexpr (NL > 0) nlines = NL;
  const int nstrips = (ncols + CW - 1) / CW;
  const int item = blockIdx.x;  // (line set j, strip)
  const int j = item / nstrips, strip = item - j * nstrips;
  // the z pass's symbol tables (constant) behind the strip buffer: lambda
  // along the lines, and lambda and the Parseval weight of the strip's columns
  T* LL = reinterpret_cast<T*>(smem + (size_t)nlines * CW * sizeof(cx<T>));
  T* LC = LL + nlines;
  T* WC = LC + CW;
  if (stage == 1 && sp.laml) {
    for (int i = threadIdx.x; i < nlines; i += bd) LL[i] = sp.laml[i];
    const int c = threadIdx.x, xc = strip * CW + c;
    if (c < CW) {
      LC[c] = xc < ncols ? sp.lamc[xc] : T(0);
      WC[c] = xc < ncols ? sp.wcol[xc] : T(0);
    }
  }
  grid_dep_sync();  // plan and tables are constant; everything below follows the previous kernel
  if (sc && !col_active(mode, pmode ? pmode + b : nullptr, sc + b)) return;
  if (stage == 1 && mode == COL_ITER && pmode && pmode[b] == 1) mode = COL_TRUE;  // reliable update
  __shared__ double red[32];
  __shared__ float redf[64];
  cx<T>* B = reinterpret_cast<cx<T>*>(smem);
  cx<T>* Sj = S + (size_t)b * sst + (size_t)j * set_stride;
  const bool store = stage != 1 || (mode != COL_NORM && mode != COL_TRUENORM);
  const int x0 = strip * CW;
  const int nc = min(CW, ncols - x0);
  // shared rows: ncs columns; a compile-time plan always transforms CWC
  // columns (those past nc are zero and never stored or summed)
  const int ncs = NL > 0 ? CWC : nc;
  const int n = nlines * ncs;
  const FastDiv dc(ncs);
#pragma unroll 1
  for (int i = threadIdx.x; i < n; i += 8 * bd) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * bd;
      if (ii < n) {
        const int y = NL > 0 ? ii / (CWC > 0 ? CWC : 1) : dc.div(ii), c = ii - y * ncs;
        t[k] = c < nc ? Sj[(size_t)y * line_stride + x0 + c] : mk(T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * bd < n) B[i + k * bd] = t[k];
  }
  __syncthreads();
  Acc<T> acc;
  if constexpr (NL > 0) {
    if (stage == 2) {
      fftc<T, 1, NL, true, CWC, kLineThreads>(B, pl_s.tw, CWC);
    } else if (stage == 1) {
      // z pass: the multiplier and the Parseval sum on the last forward
      // pass's outputs, then the inverse transform
      const T m0 = sp.m0b ? (T)sp.m0b[b] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[b] : sp.m1_t;
      ZMul<T> mul{LC, WC, LL, sp.lamj[j], m0, m1, sp.invN_t, store, T(0), 0, &acc};
      fftc<T, -1, NL, true, CWC, kLineThreads>(B, pl_s.tw, CWC, mul);
      acc.add(mul.part);
      if (store) {
        __syncthreads();
        fftc<T, 1, NL, true, CWC, kLineThreads>(B, pl_s.tw, CWC);
      }
    } else {
      fftc<T, -1, NL, true, CWC, kLineThreads>(B, pl_s.tw, CWC);
    }
  } else {
    if (stage == 2) fft_lines<T, 1, FL>(B, pl_s, nc, 1, nc, true);
    else fft_lines<T, -1, FL>(B, pl_s, nc, 1, nc, true);
  }
  if (stage == 1 && NL == 0) {
    const T m0 = sp.m0b ? (T)sp.m0b[b] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[b] : sp.m1_t;
    const T invN = sp.invN_t;
    const T lj = sp.lamj[j];
    T part = T(0);
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += bd) {
      const int kl = dc.div(i), c = i - kl * ncs;
      if (c >= nc) continue;
      const T den = m0 + m1 * (LC[c] + lj + LL[kl]);
      T m;
      if constexpr (sizeof(T) == 4) m = den > T(0) ? __fdividef(1.0f, den) : T(0);
      else m = den > T(0) ? T(1) / den : T(0);
      const cx<T> w = B[i];
      part += WC[c] * m * (w.re * w.re + w.im * w.im);
      if (++cnt == 16) { acc.add(part); part = T(0); cnt = 0; }
      if (store) B[i] = scal(w, m * invN);
    }
    acc.add(part);
    if (store) {
      __syncthreads();
      fft_lines<T, 1, FL>(B, pl_s, nc, 1, nc, true);
    }
  }
  if (store) {
    for (int i = threadIdx.x; i < n; i += bd) {
      const int y = NL > 0 ? i / (CWC > 0 ? CWC : 1) : dc.div(i), c = i - y * ncs;
      if (c < nc) Sj[(size_t)y * line_stride + x0 + c] = B[i];
    }
  }
  if (stage != 1) return;
  const double bt[1] = {acc.block_total(redf, red)};
  double* part_b = partials + (size_t)b * gridDim.x;
  if (publish_partials<1>(bt, part_b, &sc[b].cnt[1])) {
    double tot[1];
    gather_partials<1>(tot, part_b, &sc[b].cnt[1], red);
    if (threadIdx.x == 0) finalize_col(sc + b, mode, tot[0] * sp.invN, pmode ? pmode + b : nullptr);
  }
}

// ---------------------------------------------------------------- launchers

template <typename T, int D, int FX>
cudaError_t launch3_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const Shape3& sh,
                             int zero_u, int filter, cudaStream_t st) {
  const int R = sh.ry_res, Z = sh.zc_res;
  const size_t sm = Row3Layout(op.nx, R, 8, (int)sizeof(T), D).total + tw_smem_bytes<T>(op.nx);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k3_residual<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.ny + R - 1) / R) * ((op.nz + Z - 1) / Z), sh.batch);
  return launch_dep(k3_residual<T, D, FX>, grid, dim3(sh.thr_res), sm, st, op, v, px, R, Z, sh.sst, zero_u,
                    filter);
}

template <typename T, int FL, int NL, int CWC>
cudaError_t launch3_lines(cx<T>* S, const Shape3& sh, int D, int axis, int stage, const FftPlanDev<T>& pl,
                          const Spec<T>& sp, int mode, double* partials, SolverScalars* sc, int* pmode,
                          cudaStream_t st) {
  const int nx = sh.nx, ny = sh.ny, nz = sh.nz;
  const int nxs = nxs_of(nx, D);
  const int CW = axis == 1 ? sh.cw_y : sh.cw_z;
  const int thr = axis == 1 ? sh.thr_y : sh.thr_z;
  const int nl = axis == 1 ? ny : nz;
  const int nset = axis == 1 ? nz : ny;
  const long long set_stride = axis == 1 ? (long long)ny * nxs : nxs;
  const long long line_stride = axis == 1 ? nxs : (long long)ny * nxs;
  const size_t sm = (size_t)nl * CW * sizeof(cx<T>) + tw_smem_bytes<T>(nl) + (size_t)(nl + 2 * CW) * sizeof(T);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k3_lines<T, FL, NL, CWC>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(nset * ((nxs + CW - 1) / CW), sh.batch);
  return launch_dep(k3_lines<T, FL, NL, CWC>, grid, dim3(NL > 0 ? kLineThreads : thr), sm, st, S, sh.sst, nset,
                    set_stride, nl, line_stride, nxs, pl, sp, CW, stage, mode, partials, sc, pmode);
}

#define FFTMECH_INST3_TD(T, D, F)                                                                    \
  template cudaError_t launch3_residual<T, D, F>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&, \
                                                 const Shape3&, int, int, cudaStream_t);
#define FFTMECH_INST3_T(T, F)                                                                        \
  FFTMECH_INST3_TD(T, 1, F)                                                                          \
  FFTMECH_INST3_TD(T, 3, F)                                                                          \
  template cudaError_t launch3_lines<T, F, 0, 0>(cx<T>*, const Shape3&, int, int, int, const FftPlanDev<T>&, \
                                           const Spec<T>&, int, double*, SolverScalars*, int*,  \
                                           cudaStream_t);
// y / z line passes of a compile-time length (float, strips of 16 columns)
#define FFTMECH_INST3_LINES_FIXED(NL)                                                                      \
  template cudaError_t launch3_lines<float, FAM_ALL, NL, 16>(cx<float>*, const Shape3&, int, int, int,    \
                                                             const FftPlanDev<float>&, const Spec<float>&, \
                                                             int, double*, SolverScalars*, int*,    \
                                                             cudaStream_t);
#define FFTMECH_INST3_FAMILY(F) \
  FFTMECH_INST3_T(float, F)     \
  FFTMECH_INST3_T(double, F)

}  // namespace fftmech
