// 3D kernels of the FFT-Galerkin preconditioned CG (potential form) on the
// grid [nz][ny][nx], x fastest.
//
// The operator, multiplier and PCG recursion are those of the 2D kernels
// with a third direction: K u = grad+^T [g C : sym grad+ u] for the three
// displacement components (D = 3), or K u = c0 u + grad+^T [kap grad+ u]
// for a scalar (D = 1); the preconditioner is 1 / (m0 + m1 |D|^2) with
// |D|^2 = lam_x + lam_y + lam_z (the forward-difference symbol of Sec. 2.6
// in the projection of App. A, Eq. g-42).
//
// One PCG iteration is five launches:
//   direction (x lines): z = x-IFFT(S); p = z + beta p_old; <p, K p>
//   update    (x lines): u += alpha p; r -= alpha K p; S = x-FFT(r)
//   y pass    (y lines): S = y-FFT(S)
//   z pass    (z lines): S = z-IFFT(m(k) z-FFT(S)); <r, M^-1 r>
//   y pass    (y lines): S = y-IFFT(S)
// Spectral rows: row (z, y) of S holds, for D = 3, the packed components
// (r_x + i r_y) as nx complex numbers followed by the half spectrum
// (nx/2 + 1 numbers) of r_z; for D = 1 only the half spectrum. A real line's
// spectrum is Hermitian, so the other half is never stored or transformed
// along y and z; the x-IFFT rebuilds it.
//
// The x-line kernels take a brick of R lines in y and march through Zc
// planes in z, keeping two planes of the direction and of the stress (or
// flux) components that are differenced along z in shared memory, so each
// plane is read once per brick plus one halo plane.
#pragma once

#include <type_traits>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

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

// Direction (KIND 0) or FP64 iterate (KIND 1) of plane z (periodic) into
// ring slot s of P: lines y0 - 1 .. y0 + W - 2 of every component.
template <typename T, typename CT, int D, int KIND>
__device__ __forceinline__ void load_plane3(CT* P, const Op<T>& op, const Vec2<T>& v, int z, int s, int y0, int W,
                                            size_t PS, size_t N, int zero_u) {
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const int zw = wrap_z(z, nz);
  CT* dst = P + (size_t)s * D * PS;
  if constexpr (KIND == 0) {
#pragma unroll
    for (int c = 0; c < D; ++c) g2s_rows<4>(dst + c * PS, v.p_in + c * N + (size_t)zw * plane, y0 - 1, W, nx, ny);
  } else {
    const FastDiv dnx(nx);
    for (int i = threadIdx.x; i < W * nx; i += blockDim.x) {
      const int l = dnx.div(i), x = i - l * nx;
      const size_t gi = (size_t)zw * plane + (size_t)wrap_y(y0 - 1 + l, ny) * nx + x;
      const bool keep = (D == 1) && op.mask && op.mask[gi];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double val;
        if constexpr (sizeof(T) == 4) val = (double)v.uh[c * N + gi] + (double)v.ul[c * N + gi];
        else val = v.u[c * N + gi];
        if (zero_u && !keep) val = 0.0;
        dst[c * PS + i] = val;
      }
    }
  }
}

// ---------------------------------------------------------------- stencil rows
// KIND 0 (update): u += alpha p; r -= alpha K p; S = x-FFT(r), in T.
// KIND 1 (residual): r = b - K u in FP64 from the iterate (zero_u: u = 0
// except on Dirichlet voxels; filter: only problems with a nonzero mode),
// written as T; S = x-FFT(r).
// Plane loop: zz = z0 - 1 (halo: z-differenced stress only) .. z0 + planes - 1.
template <typename T, int D, int FX, int KIND>
__global__ void FFTMECH_BOUNDS3 k3_rows(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R, int Zc, long long sst,
                                        int zero_u, int filter) {
  using CT = typename std::conditional<KIND == 1, double, T>::type;
  using C = Comp3<D>;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  if (KIND == 1 && filter && !(v.mode && v.mode[bp] != 0)) return;
  problem_views3<T, D>(op, v, bp, N, sst);
  int u_only = 0;
  double alpha = 0.0;  // FP64 path
  float ah = 0.f, al = 0.f;  // MIXED: alpha = ah + al
  if constexpr (KIND == 0) {
    u_only = v.mode ? (v.mode[bp] == 1) : 0;
    if (done_flag(v.sc)) return;
    if constexpr (sizeof(T) == 4) {
      ah = vol_readf(&v.sc->alpha_h);
      al = vol_readf(&v.sc->alpha_l);
    } else {
      alpha = vol_read(&v.sc->alpha);
    }
  }
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  const int nty = (ny + R - 1) / R;
  const int tz = blockIdx.x / nty, ty = blockIdx.x - tz * nty;
  const int y0 = ty * R, rows = min(R, ny - y0);
  const int z0 = tz * Zc, planes = min(Zc, nz - z0);
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nxa = D == 3 ? nx : 0, nxh = nx / 2 + 1, nxs = nxa + nxh;
  if constexpr (KIND == 0) {
    if (u_only) {  // reliable-update iteration: only the iterate moves
      for (int zz = z0; zz < z0 + planes; ++zz) {
        const size_t t0 = (size_t)zz * plane + (size_t)y0 * nx;
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
      }
      return;
    }
  }
  const Row3Layout L(nx, R, (int)sizeof(CT), (int)sizeof(T), D, KIND);
  CT* P = reinterpret_cast<CT*>(smem + L.P);
  CT* SP = reinterpret_cast<CT*>(smem + L.SP);
  CT* SZ = reinterpret_cast<CT*>(smem + L.SZ);
  CT* RS = reinterpret_cast<CT*>(smem + L.RS);
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + L.F);
  T* MG = reinterpret_cast<T*>(smem + L.MG);
  uint8_t* PH = smem + L.PH;
  uint8_t* MK = smem + L.MK;
  const int W = rows + 2;                   // direction lines y0 - 1 .. y0 + rows
  const size_t PS = (size_t)(R + 2) * nx;   // one component of one P slot
  const size_t SS = (size_t)(R + 1) * nx;   // one stress component of one plane
  const T* matg = (D == 3) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  // KIND 0 computes in T with the host-rounded constants; KIND 1 in FP64
  const CT ih = KIND == 0 ? (CT)op.ih_t : (CT)(1.0 / op.h);
  const CT lam0 = KIND == 0 ? (CT)op.lam_t[0] : (CT)op.lam[0], lam1 = KIND == 0 ? (CT)op.lam_t[1] : (CT)op.lam[1];
  const CT mu0 = KIND == 0 ? (CT)op.mu_t[0] : (CT)op.mu[0], mu1 = KIND == 0 ? (CT)op.mu_t[1] : (CT)op.mu[1];
  const CT kap0 = KIND == 0 ? (CT)op.kap_t[0] : (CT)op.kap[0], kap1 = KIND == 0 ? (CT)op.kap_t[1] : (CT)op.kap[1];
  const CT c0c = KIND == 0 ? (CT)op.c0c_t : (CT)op.c0c;
  const CT a = sizeof(T) == 4 ? (CT)ah : (CT)alpha;
  const FastDiv dnx(nx);

  load_plane3<T, CT, D, KIND>(P, op, v, z0 - 1, 0, y0, W, PS, N, zero_u);
  for (int zz = z0 - 1; zz < z0 + planes; ++zz) {
    const int cur = (zz - z0 + 1) & 1, nxt = cur ^ 1;
    const bool inner = zz >= z0;
    const int zw = wrap_z(zz, nz);
    const size_t pz = (size_t)zw * plane;
    load_plane3<T, CT, D, KIND>(P, op, v, zz + 1, nxt, y0, W, PS, N, zero_u);
    if (matg) g2s_rows<4>(MG, matg + pz, y0 - 1, rows + 1, nx, ny);
    g2s_rows<4>(PH, op.phase + pz, y0 - 1, rows + 1, nx, ny);
    if (inner) {
      if constexpr (KIND == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) g2s_vec<4, false>(RS + (size_t)c * rows * nx, v.r + c * N + pz + (size_t)y0 * nx, rows * nx);
      }
      if (masked) g2s_vec<4, true>(MK, op.mask + pz + (size_t)y0 * nx, rows * nx);
    }
    __syncthreads();
    const CT* Pc = P + (size_t)cur * D * PS;
    const CT* Pn = P + (size_t)nxt * D * PS;
    CT* Zc_ = SZ + (size_t)cur * C::NZ * SS;
    const CT* Zp = SZ + (size_t)nxt * C::NZ * SS;  // previous plane (same slot parity as the next)
    if constexpr (KIND == 0) {
      if (inner) {  // iterate update on the interior lines of this plane
        const size_t t0 = pz + (size_t)y0 * nx;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int c = 0; c < D; ++c)
            df_axpy_g<4>(v.uh + c * N + t0, v.ul + c * N + t0, Pc + c * PS + nx, ah, al, rows * nx);
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) axpy_g<4>(v.u + c * N + t0, Pc + c * PS + nx, alpha, rows * nx);
        }
      }
    }
    // stress / flux of plane zz at lines y0 - 1 .. y0 + rows - 1
    for (int i = tid; i < (rows + 1) * nx; i += bd) {
      const int l = dnx.div(i), x = i - l * nx;
      const int xp = (x + 1 == nx) ? 0 : x + 1;
      const int ix = l * nx + xp;
      const bool sol = PH[i] != 0;
      if constexpr (D == 3) {
        const CT* Ux = Pc;
        const CT* Uy = Pc + PS;
        const CT* Uz = Pc + 2 * PS;
        const CT ux = Ux[i], uy = Uy[i], uz = Uz[i];
        CT exx = (Ux[ix] - ux) * ih;
        CT eyy = (Uy[i + nx] - uy) * ih;
        CT ezz = (Pn[2 * PS + i] - uz) * ih;
        CT eyz = CT(0.5) * ((Pn[PS + i] - uy) + (Uz[i + nx] - uz)) * ih;
        CT exz = CT(0.5) * ((Pn[i] - ux) + (Uz[ix] - uz)) * ih;
        CT exy = CT(0.5) * ((Ux[i + nx] - ux) + (Uy[ix] - uy)) * ih;
        if constexpr (KIND == 1) {
          const size_t gi = pz + (size_t)wrap_y(y0 - 1 + l, ny) * nx + x;
          const double e = op.eig ? (double)op.eig[gi] : 0.0;
          exx += op.E[0] - e;
          eyy += op.E[1] - e;
          ezz += op.E[2] - e;
          eyz += op.E[3];
          exz += op.E[4];
          exy += op.E[5];
        }
        const CT gg = matg ? (CT)MG[i] : CT(1);
        const CT lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
        const CT lt = lam * (exx + eyy + ezz);
        const CT m2 = CT(2) * mu;
        if (inner) {
          SP[i] = lt + m2 * exx;
          SP[SS + i] = lt + m2 * eyy;
          SP[2 * SS + i] = m2 * exy;
        }
        Zc_[i] = m2 * exz;
        Zc_[SS + i] = m2 * eyz;
        Zc_[2 * SS + i] = lt + m2 * ezz;
      } else {
        const CT p = Pc[i];
        const CT kap = sol ? kap1 : kap0;
        CT gx = (Pc[ix] - p) * ih, gy = (Pc[i + nx] - p) * ih, gz = (Pn[i] - p) * ih;
        if constexpr (KIND == 1) {
          gx += op.G[0];
          gy += op.G[1];
          gz += op.G[2];
        }
        if (inner) {
          SP[i] = kap * gx;
          SP[SS + i] = kap * gy;
        }
        Zc_[i] = kap * gz;
      }
    }
    __syncthreads();
    if (!inner) continue;
    // K p (or the residual) on the interior lines, packed for the x transform
    for (int i = tid; i < rows * nx; i += bd) {
      const int lr = dnx.div(i), x = i - lr * nx;
      const int l = lr + 1;
      const int xm = (x == 0) ? nx - 1 : x - 1;
      const int c = l * nx + x, cxm = l * nx + xm;
      const size_t gi = pz + (size_t)(y0 + lr) * nx + x;
      if constexpr (D == 3) {
        const CT* Sxx = SP;
        const CT* Syy = SP + SS;
        const CT* Sxy = SP + 2 * SS;
        const CT* Sxz = Zc_;
        const CT* Syz = Zc_ + SS;
        const CT* Szz = Zc_ + 2 * SS;
        const CT q0 = ((Sxx[cxm] - Sxx[c]) + (Sxy[c - nx] - Sxy[c]) + (Zp[c] - Sxz[c])) * ih;
        const CT q1 = ((Sxy[cxm] - Sxy[c]) + (Syy[c - nx] - Syy[c]) + (Zp[SS + c] - Syz[c])) * ih;
        const CT q2 = ((Sxz[cxm] - Sxz[c]) + (Syz[c - nx] - Syz[c]) + (Zp[2 * SS + c] - Szz[c])) * ih;
        T r0, r1, r2;
        if constexpr (KIND == 0) {
          r0 = RS[i] - a * q0;
          r1 = RS[rows * nx + i] - a * q1;
          r2 = RS[2 * rows * nx + i] - a * q2;
        } else {
          r0 = (T)(-q0);
          r1 = (T)(-q1);
          r2 = (T)(-q2);
        }
        v.r[gi] = r0;
        v.r[N + gi] = r1;
        v.r[2 * N + gi] = r2;
        F[i] = mk(r0, r1);
        F[(size_t)rows * nx + i] = mk(r2, T(0));
      } else {
        const CT* Jx = SP;
        const CT* Jy = SP + SS;
        const CT div = ((Jx[cxm] - Jx[c]) + (Jy[c - nx] - Jy[c]) + (Zp[c] - Zc_[c])) * ih;
        const CT c0v = c0c + (matg ? (CT)MG[c] : CT(0));
        T r0;
        if constexpr (KIND == 0) {
          CT q = c0v * Pc[c] + div;
          if (masked && MK[i]) q = CT(0);
          r0 = RS[i] - a * q;
        } else {
          const double src = op.srcd ? op.srcd[gi] : (op.srct ? (double)op.srct[gi] : 0.0);
          double rr = op.src_scale * src - (double)c0v * Pc[c] - div;
          if (op.mask && op.mask[gi]) rr = 0.0;
          r0 = (T)rr;
        }
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

// p of plane z (periodic) on lines y0 .. y0 + rows into ring slot s:
// x-IFFT of the spectral rows (the real field's other half spectrum rebuilt
// by conjugate symmetry), p = z + beta p_old; stored if z < z_end.
template <typename T, int D, int FX>
__device__ __forceinline__ void make_p3(cx<T>* F, T* P, uint8_t* MK, const Op<T>& op, const Vec2<T>& v,
                                        const FftPlanDev<T>& px, int z, int s, int z_end, int y0, int rows, int R,
                                        bool with_old, T b, size_t N) {
  using C = Comp3<D>;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const int nxa = D == 3 ? nx : 0, nxh = nx / 2 + 1, nxs = nxa + nxh;
  const int W = rows + 1;
  const size_t PS = (size_t)(R + 1) * nx;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int zw = wrap_z(z, nz);
  const bool own = z < z_end;
  const bool masked = (D == 1) && op.mask;
  T* Ps = P + (size_t)s * D * PS;
  cx<T>* FB = F + (size_t)(C::NF - 1) * W * nx;  // the real field's lines
  for (int l = 0; l < W; ++l) {
    const cx<T>* Srow = v.S + ((size_t)zw * ny + wrap_y(y0 + l, ny)) * nxs;
    if constexpr (D == 3) g2s_vec<4, true>(F + (size_t)l * nx, Srow, nx);
    g2s_vec<4, true>(FB + (size_t)l * nx, Srow + nxa, nxh);
  }
  if (with_old) {
#pragma unroll
    for (int c = 0; c < D; ++c) g2s_rows<4>(Ps + c * PS, v.p_in + c * N + (size_t)zw * plane, y0, W, nx, ny);
  }
  if (masked) g2s_rows<4>(MK, op.mask + (size_t)zw * plane, y0, W, nx, ny);
  __syncthreads();
  // the other half of each real line's spectrum: X(nx - k) = conj X(k)
  const int nup = nx - nxh;
  for (int i = tid; i < W * nup; i += bd) {
    const int l = i / nup, k = nxh + (i - l * nup);
    const cx<T> w = FB[(size_t)l * nx + (nx - k)];
    FB[(size_t)l * nx + k] = mk(w.re, -w.im);
  }
  __syncthreads();
  fft_lines_call<T, 1, FX>(F, px, C::NF * W, nx, 1, false);
  const FastDiv dnx(nx);
  for (int i = tid; i < W * nx; i += bd) {
    const int l = dnx.div(i);
    if constexpr (D == 3) {
      const cx<T> zA = F[i];
      T p0 = zA.re, p1 = zA.im, p2 = FB[i].re;
      if (with_old) {
        p0 += b * Ps[i];
        p1 += b * Ps[PS + i];
        p2 += b * Ps[2 * PS + i];
      }
      Ps[i] = p0;
      Ps[PS + i] = p1;
      Ps[2 * PS + i] = p2;
      if (own && l < rows) {
        const size_t gi = (size_t)zw * plane + (size_t)y0 * nx + i;
        v.p_out[gi] = p0;
        v.p_out[N + gi] = p1;
        v.p_out[2 * N + gi] = p2;
      }
    } else {
      T p0 = FB[i].re;
      if (masked && MK[i]) p0 = T(0);
      if (with_old) p0 += b * Ps[i];
      Ps[i] = p0;
      if (own && l < rows) v.p_out[(size_t)zw * plane + (size_t)y0 * nx + i] = p0;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- direction
// z = x-IFFT(S) on lines y0 .. y0 + rows (one halo line) of planes
// z0 .. z0 + planes (one halo plane); p = z + beta p_old; <p, K p> as the
// sum of the energy density over the brick.
template <typename T, int D, int FX>
__global__ void FFTMECH_BOUNDS3 k3_direction(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int R, int Zc,
                                             long long sst) {
  using C = Comp3<D>;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  problem_views3<T, D>(op, v, bp, N, sst);
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
  const bool with_old = b != T(0);  // the first iteration has p = z
  const int nty = (ny + R - 1) / R;
  const int tz = blockIdx.x / nty, ty = blockIdx.x - tz * nty;
  const int y0 = ty * R, rows = min(R, ny - y0);
  const int z0 = tz * Zc, planes = min(Zc, nz - z0);
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nxa = D == 3 ? nx : 0, nxh = nx / 2 + 1, nxs = nxa + nxh;
  const int W = rows + 1;
  const Dir3Layout L(nx, R, (int)sizeof(T), D);
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + L.F);
  T* P = reinterpret_cast<T*>(smem + L.P);
  T* MG = reinterpret_cast<T*>(smem + L.MG);
  uint8_t* PH = smem + L.PH;
  uint8_t* MK = smem + L.MK;
  const size_t PS = (size_t)(R + 1) * nx;
  const T* matg = (D == 3) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  const FastDiv dnx(nx);
  cx<T>* FB = F + (size_t)(C::NF - 1) * W * nx;  // the real field's lines

  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  Acc<T> acc;
  make_p3<T, D, FX>(F, P, MK, op, v, px_s, z0, 0, z0 + planes, y0, rows, R, with_old, b, N);
  for (int zz = z0; zz < z0 + planes; ++zz) {
    const int cur = (zz - z0) & 1, nxt = cur ^ 1;
    make_p3<T, D, FX>(F, P, MK, op, v, px_s, zz + 1, nxt, z0 + planes, y0, rows, R, with_old, b, N);
    const size_t t0 = (size_t)zz * plane + (size_t)y0 * nx;
    if (matg) g2s_vec<4, true>(MG, matg + t0, rows * nx);
    g2s_vec<4, true>(PH, op.phase + t0, rows * nx);
    __syncthreads();
    const T* Pc = P + (size_t)cur * D * PS;
    const T* Pn = P + (size_t)nxt * D * PS;
    T part = T(0);
    int cnt = 0;
    for (int i = tid; i < rows * nx; i += bd) {
      const int l = dnx.div(i), x = i - l * nx;
      const int ix = l * nx + ((x + 1 == nx) ? 0 : x + 1);
      const bool sol = PH[i] != 0;
      T w;
      if constexpr (D == 3) {
        const T* Ux = Pc;
        const T* Uy = Pc + PS;
        const T* Uz = Pc + 2 * PS;
        const T ux = Ux[i], uy = Uy[i], uz = Uz[i];
        const T exx = (Ux[ix] - ux) * ih;
        const T eyy = (Uy[i + nx] - uy) * ih;
        const T ezz = (Pn[2 * PS + i] - uz) * ih;
        const T eyz = T(0.5) * ((Pn[PS + i] - uy) + (Uz[i + nx] - uz)) * ih;
        const T exz = T(0.5) * ((Pn[i] - ux) + (Uz[ix] - uz)) * ih;
        const T exy = T(0.5) * ((Ux[i + nx] - ux) + (Uy[ix] - uy)) * ih;
        const T gg = matg ? MG[i] : T(1);
        const T lam = sol ? lam1 : lam0, mu = sol ? mu1 : mu0;
        const T tr = exx + eyy + ezz;
        w = gg * (lam * tr * tr +
                  T(2) * mu * (exx * exx + eyy * eyy + ezz * ezz + T(2) * (exy * exy + exz * exz + eyz * eyz)));
      } else {
        const T p = Pc[i];
        const T gx = (Pc[ix] - p) * ih, gy = (Pc[i + nx] - p) * ih, gz = (Pn[i] - p) * ih;
        const T c0v = c0c + (matg ? MG[i] : T(0));
        w = c0v * p * p + (sol ? kap1 : kap0) * (gx * gx + gy * gy + gz * gz);
      }
      part += w;  // non-negative terms
      if (++cnt == 16) { acc.add(part); part = T(0); cnt = 0; }
    }
    acc.add(part);
    __syncthreads();
  }
  const double bt[1] = {acc.block_total(redf, red)};
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- line passes
// A strip of CW spectral columns of one line set: nlines complex numbers per
// column, line_stride apart. Line set j of problem b starts at
// S + b sst + j set_stride (y pass: j = z plane; z pass: j = ky).
// stage 0 / 2: forward / inverse FFT along the lines (y pass).
// stage 1 (z pass): forward FFT, multiply by m(k) / N with
//   lambda = lamc[column] + lamj[j] + laml[line], sum of wcol m |S|^2
//   (Parseval over the full spectrum: the half-spectrum columns count
//   twice except kx = 0 and kx = nx/2), inverse FFT unless NORM/TRUENORM.
template <typename T, int FL>
__global__ void FFTMECH_BOUNDS3 k3_lines(cx<T>* S, long long sst, int nset, long long set_stride, int nlines,
                                         long long line_stride, int ncols, FftPlanDev<T> pl, Spec<T> sp,
                                         int CW, int stage, int mode, double* partials, SolverScalars* sc,
                                         const int* pmode) {
  const int bpj = blockIdx.y;
  const int b = bpj / nset, j = bpj - b * nset;
  if (sc && !col_active(mode, pmode ? pmode + b : nullptr, sc + b)) return;
  if (stage == 1 && mode == COL_ITER && pmode && pmode[b] == 1) mode = COL_TRUE;  // reliable update
  S += (size_t)b * sst + (size_t)j * set_stride;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(pl.n);
  const FftPlanDev<T> pl_s = plan_to_smem(pl, reinterpret_cast<cx<T>*>(smem_all));
  __shared__ double red[32];
  __shared__ float redf[64];
  cx<T>* B = reinterpret_cast<cx<T>*>(smem);
  const int x0 = blockIdx.x * CW;
  const int nc = min(CW, ncols - x0);
  const int n = nlines * nc;
  const int bd = blockDim.x;
  const FastDiv dc(nc);
  for (int i = threadIdx.x; i < n; i += 8 * bd) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * bd;
      if (ii < n) {
        const int y = dc.div(ii), c = ii - y * nc;
        t[k] = S[(size_t)y * line_stride + x0 + c];
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * bd < n) B[i + k * bd] = t[k];
  }
  __syncthreads();
  if (stage == 2) fft_lines<T, 1, FL>(B, pl_s, nc, 1, nc, true);
  else fft_lines<T, -1, FL>(B, pl_s, nc, 1, nc, true);
  const bool store = stage != 1 || (mode != COL_NORM && mode != COL_TRUENORM);
  Acc<T> acc;
  if (stage == 1) {
    const T m0 = sp.m0b ? (T)sp.m0b[b] : sp.m0_t, m1 = sp.m1b ? (T)sp.m1b[b] : sp.m1_t;
    const T invN = sp.invN_t;
    const T lj = sp.lamj[j];
    T part = T(0);
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += bd) {
      const int kl = dc.div(i), c = i - kl * nc;
      const T den = m0 + m1 * (sp.lamc[x0 + c] + lj + sp.laml[kl]);
      T m;
      if constexpr (sizeof(T) == 4) m = den > T(0) ? __fdividef(1.0f, den) : T(0);
      else m = den > T(0) ? T(1) / den : T(0);
      const cx<T> w = B[i];
      part += sp.wcol[x0 + c] * m * (w.re * w.re + w.im * w.im);
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
      const int y = dc.div(i), c = i - y * nc;
      S[(size_t)y * line_stride + x0 + c] = B[i];
    }
  }
  if (stage != 1) return;
  const double bt[1] = {acc.block_total(redf, red)};
  double* part_b = partials + (size_t)b * nset * gridDim.x;
  const int slot = j * gridDim.x + blockIdx.x, total = nset * gridDim.x;
  if (publish_partials_at<1>(bt, part_b, slot, total, &sc[b].cnt[1])) {
    double tot[1];
    gather_partials_n<1>(tot, part_b, total, &sc[b].cnt[1], red);
    if (threadIdx.x == 0) finalize_col(sc + b, mode, tot[0] * sp.invN);
  }
}

// ---------------------------------------------------------------- launchers
template <typename K>
static cudaError_t set_smem3(K kernel, size_t bytes, int& configured) {
  if (configured) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if ((long long)bytes > (long long)dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e == cudaSuccess) configured = 1;
  return e;
}

template <typename T, int D, int FX>
cudaError_t launch3_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const Shape3& sh,
                             int zero_u, int filter, cudaStream_t st) {
  const int R = sh.ry_res, Z = sh.zc_res;
  const size_t sm = Row3Layout(op.nx, R, 8, (int)sizeof(T), D, 1).total + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem3(k3_rows<T, D, FX, 1>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.ny + R - 1) / R) * ((op.nz + Z - 1) / Z), sh.batch);
  k3_rows<T, D, FX, 1><<<grid, sh.thr_res, sm, st>>>(op, v, px, R, Z, sh.sst, zero_u, filter);
  return cudaGetLastError();
}

template <typename T, int D, int FX>
cudaError_t launch3_update(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const Shape3& sh,
                           cudaStream_t st) {
  const int R = sh.ry_upd, Z = sh.zc_upd;
  const size_t sm = Row3Layout(op.nx, R, (int)sizeof(T), (int)sizeof(T), D, 0).total + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem3(k3_rows<T, D, FX, 0>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.ny + R - 1) / R) * ((op.nz + Z - 1) / Z), sh.batch);
  k3_rows<T, D, FX, 0><<<grid, sh.thr_upd, sm, st>>>(op, v, px, R, Z, sh.sst, 0, 0);
  return cudaGetLastError();
}

template <typename T, int D, int FX>
cudaError_t launch3_direction(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const Shape3& sh,
                              cudaStream_t st) {
  const int R = sh.ry_dir, Z = sh.zc_dir;
  const size_t sm = Dir3Layout(op.nx, R, (int)sizeof(T), D).total + tw_smem_bytes<T>(op.nx);
  static int cfg = 0;
  cudaError_t e = set_smem3(k3_direction<T, D, FX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.ny + R - 1) / R) * ((op.nz + Z - 1) / Z), sh.batch);
  k3_direction<T, D, FX><<<grid, sh.thr_dir, sm, st>>>(op, v, px, R, Z, sh.sst);
  return cudaGetLastError();
}

template <typename T, int FL>
cudaError_t launch3_lines(cx<T>* S, const Shape3& sh, int D, int axis, int stage, const FftPlanDev<T>& pl,
                          const Spec<T>& sp, int mode, double* partials, SolverScalars* sc, const int* pmode,
                          cudaStream_t st) {
  const int nx = sh.nx, ny = sh.ny, nz = sh.nz;
  const int nxs = nxs_of(nx, D);
  const int CW = axis == 1 ? sh.cw_y : sh.cw_z;
  const int thr = axis == 1 ? sh.thr_y : sh.thr_z;
  const int nl = axis == 1 ? ny : nz;
  const int nset = axis == 1 ? nz : ny;
  const long long set_stride = axis == 1 ? (long long)ny * nxs : nxs;
  const long long line_stride = axis == 1 ? nxs : (long long)ny * nxs;
  const size_t sm = (size_t)nl * CW * sizeof(cx<T>) + tw_smem_bytes<T>(nl);
  static int cfg = 0;
  cudaError_t e = set_smem3(k3_lines<T, FL>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((nxs + CW - 1) / CW, sh.batch * nset);
  k3_lines<T, FL><<<grid, thr, sm, st>>>(S, sh.sst, nset, set_stride, nl, line_stride, nxs, pl, sp, CW, stage, mode,
                                         partials, sc, pmode);
  return cudaGetLastError();
}

#define FFTMECH_INST3_TD(T, D, F)                                                                    \
  template cudaError_t launch3_residual<T, D, F>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&, \
                                                 const Shape3&, int, int, cudaStream_t);           \
  template cudaError_t launch3_update<T, D, F>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&,   \
                                               const Shape3&, cudaStream_t);                       \
  template cudaError_t launch3_direction<T, D, F>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&, \
                                                  const Shape3&, cudaStream_t);
#define FFTMECH_INST3_T(T, F)                                                                        \
  FFTMECH_INST3_TD(T, 1, F)                                                                          \
  FFTMECH_INST3_TD(T, 3, F)                                                                          \
  template cudaError_t launch3_lines<T, F>(cx<T>*, const Shape3&, int, int, int, const FftPlanDev<T>&, \
                                           const Spec<T>&, int, double*, SolverScalars*, const int*,  \
                                           cudaStream_t);
#define FFTMECH_INST3_FAMILY(F) \
  FFTMECH_INST3_T(float, F)     \
  FFTMECH_INST3_T(double, F)

}  // namespace fftmech
