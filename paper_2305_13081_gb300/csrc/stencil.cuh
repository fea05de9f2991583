// Stencil kernels of the split PCG iteration: q = K p and the energy form
// <p, K p> = sum over voxels of eps(p) : g C : eps(p) (elasticity) or
// c0 p^2 + kap |grad+ p|^2 (scalar problems), whose last block sets
// alpha = <r, M^-1 r> / <p, K p>. K = grad+^T [g C sym grad+] (Eq. solid
// with the forward-difference gradient of Sec. 2.6) or c0 + grad+^T kap
// grad+ (Eqs. diffusion-final, crack-fft); masked voxels (Dirichlet) get
// q = 0. 2D: warps march down column strips with the stencil's neighbours
// in registers and shuffles. 3D: tiles of TX x TY voxels with a one-voxel
// halo in shared memory march through Zc planes keeping two planes of the
// direction and of the z-differenced stress (or flux) components.
#pragma once

#include <algorithm>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

template <typename T, int D>
__device__ __forceinline__ void sten_views(Op<T>& op, Vec2<T>& v, int b, size_t N) {
  const size_t o1 = (size_t)b * N, oD = (size_t)b * D * N;
  op.phase += o1;
  if (op.g) op.g += o1;
  if (op.c0f) op.c0f += o1;
  if (op.mask) op.mask += o1;
  v.p_in += oD;
  v.q += oD;
  v.sc += b;
}


// ---------------------------------------------------------------- 2D
// One warp takes a strip of kStrip2 = 30 columns and TY rows: lane l holds
// column x0 + l - 1 (lane 0 the left halo column, lane 31 the right one;
// lanes 1 .. 30 produce q). The warp first loads every value it needs (the
// direction on rows y0 - 1 .. y0 + TY, the material on rows y0 - 1 ..
// y0 + TY - 1) into registers, so a strip costs one memory round trip; then
// it walks down the rows: the right neighbour's direction and the left
// neighbour's stress (flux) come from warp shuffles, the row above's stress
// from the previous step. No shared memory and no barrier; warps take
// strips warp-stride over the grid, one reduction ticket per block.
constexpr int kStrip2 = 30;
constexpr int kSten2Threads = 256;

template <typename T, int D, int TY>
__global__ void __launch_bounds__(kSten2Threads) k_sten2(Op<T> op, Vec2<T> v) {
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  sten_views<T, D>(op, v, bp, N);
  grid_dep_sync();
  if (done_flag(v.sc)) return;
  commit_pending_rz(v.sc);
  __shared__ double red[32];
  __shared__ float redf[64];
  const T* __restrict__ P = v.p_in;
  const T* __restrict__ matg = (D == 2) ? op.g : op.c0f;
  const uint8_t* __restrict__ ph = op.phase;
  const uint8_t* __restrict__ msk = (D == 1) ? op.mask : nullptr;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  const int nsx = (nx + kStrip2 - 1) / kStrip2;
  const int items = nsx * ((ny + TY - 1) / TY);
  Acc<T> acc;
  for (int item = blockIdx.x * nwarps + (int)(threadIdx.x >> 5); item < items; item += gridDim.x * nwarps) {
    const int sy = item / nsx, sx = item - sy * nsx;
    const int x0 = sx * kStrip2, y0 = sy * TY;
    const int wx = min(kStrip2, nx - x0), wy = min(TY, ny - y0);
    const int x = (x0 - 1 + lane + nx) % nx;
    const bool own = lane >= 1 && lane <= kStrip2 && lane - 1 < wx;
    // row k of the strip is grid row y0 - 1 + k (wrapped)
    int row[TY + 2];
    row[0] = (y0 - 1 + ny) % ny;
#pragma unroll
    for (int k = 1; k < TY + 2; ++k) row[k] = row[k - 1] + 1 == ny ? 0 : row[k - 1] + 1;
    T p[TY + 2][D], g[TY + 1];
    bool sol[TY + 1], mk[TY + 1];
#pragma unroll
    for (int k = 0; k < TY + 2; ++k) {
      const size_t o = (size_t)row[k] * nx + x;
#pragma unroll
      for (int c = 0; c < D; ++c) p[k][c] = P[c * N + o];
      if (k < TY + 1) {
        sol[k] = ph[o] != 0;
        g[k] = matg ? matg[o] : T(0);
        mk[k] = msk ? msk[o] != 0 : false;
      }
    }
    T up0 = T(0), up1 = T(0);  // the row above: D = 2 (sxy, syy), D = 1 (Jy)
    T part = T(0);
#pragma unroll
    for (int k = 0; k < TY + 1; ++k) {
      const bool out = own && k >= 1 && k <= wy;
      T pr[D];
#pragma unroll
      for (int c = 0; c < D; ++c) pr[c] = __shfl_down_sync(FULL, p[k][c], 1);
      if constexpr (D == 2) {
        const T exx = (pr[0] - p[k][0]) * ih;
        const T eyy = (p[k + 1][1] - p[k][1]) * ih;
        const T exy = T(0.5) * ((p[k + 1][0] - p[k][0]) + (pr[1] - p[k][1])) * ih;
        const T gg = matg ? g[k] : T(1);
        const T lam = gg * (sol[k] ? lam1 : lam0), mu = gg * (sol[k] ? mu1 : mu0);
        const T lt = lam * (exx + eyy);
        const T sxx = lt + T(2) * mu * exx, syy = lt + T(2) * mu * eyy, sxy = T(2) * mu * exy;
        const T lxx = __shfl_up_sync(FULL, sxx, 1), lxy = __shfl_up_sync(FULL, sxy, 1);
        if (out) {
          const size_t gi = (size_t)row[k] * nx + x;
          v.q[gi] = ((lxx - sxx) + (up0 - sxy)) * ih;
          v.q[N + gi] = ((lxy - sxy) + (up1 - syy)) * ih;
          part += exx * sxx + eyy * syy + T(2) * exy * sxy;
        }
        up0 = sxy;
        up1 = syy;
      } else {
        const T pk = p[k][0];
        const T kap = sol[k] ? kap1 : kap0;
        const T gx = (pr[0] - pk) * ih, gy = (p[k + 1][0] - pk) * ih;
        const T jx = kap * gx, jy = kap * gy;
        const T ljx = __shfl_up_sync(FULL, jx, 1);
        if (out) {
          const size_t gi = (size_t)row[k] * nx + x;
          const T c0 = c0c + g[k];
          T q = c0 * pk + ((ljx - jx) + (up0 - jy)) * ih;
          if (mk[k]) q = T(0);
          v.q[gi] = q;
          part += c0 * pk * pk + kap * (gx * gx + gy * gy);
        }
        up0 = jy;
      }
    }
    acc.add(part);
  }
  double* partials = v.partials + (size_t)bp * gridDim.x;
  if (v.nsten > 0) {  // deferred: the update kernel's blocks sum the partials
    store_deferred_partial<T>(acc, partials + blockIdx.x, redf, red);
    return;
  }
  const double bt[1] = {acc.block_total(redf, red)};
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- 3D
// One warp takes a brick of kStrip2 = 30 columns (lanes 0 and 31 are halo
// columns), R rows and Zc planes, and marches through the planes from the
// halo plane z0 - 1. For each plane it walks the R + 1 rows y0 - 1 ..
// y0 + R - 1: the stress (flux) at a row needs the direction on the row, the
// row below and the next plane; x neighbours come from shuffles, the row
// above's stress from the previous row step and the previous plane's
// z-differenced components from registers kept per row.
template <typename T, int D, int R>
__global__ void __launch_bounds__(kSten2Threads) k_sten3(Op<T> op, Vec2<T> v, int Zc) {
  constexpr int NZ = D == 3 ? 3 : 1;  // z-differenced components (sxz, syz, szz) or Jz
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  sten_views<T, D>(op, v, bp, N);
  grid_dep_sync();
  if (done_flag(v.sc)) return;
  commit_pending_rz(v.sc);
  __shared__ double red[32];
  __shared__ float redf[64];
  const T* __restrict__ P = v.p_in;
  const T* __restrict__ matg = (D == 3) ? op.g : op.c0f;
  const uint8_t* __restrict__ ph = op.phase;
  const uint8_t* __restrict__ msk = (D == 1) ? op.mask : nullptr;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  const int nsx = (nx + kStrip2 - 1) / kStrip2, nsy = (ny + R - 1) / R;
  const int items = nsx * nsy * ((nz + Zc - 1) / Zc);
  Acc<T> acc;
  for (int item = blockIdx.x * nwarps + (int)(threadIdx.x >> 5); item < items; item += gridDim.x * nwarps) {
    int t = item;
    const int sx = t % nsx;
    t /= nsx;
    const int sy = t % nsy;
    const int sz = t / nsy;
    const int x0 = sx * kStrip2, y0 = sy * R, z0 = sz * Zc;
    const int wx = min(kStrip2, nx - x0), wy = min(R, ny - y0), planes = min(Zc, nz - z0);
    const int x = (x0 - 1 + lane + nx) % nx;
    const bool own = lane >= 1 && lane <= kStrip2 && lane - 1 < wx;
    size_t rowo[R + 2];  // offsets of rows y0 - 1 .. y0 + R (wrapped) within a plane
    {
      int y = (y0 - 1 + ny) % ny;
#pragma unroll
      for (int r = 0; r < R + 2; ++r) {
        rowo[r] = (size_t)y * nx + x;
        y = y + 1 == ny ? 0 : y + 1;
      }
    }
    int z = (z0 - 1 + nz) % nz;
    T pc[R + 2][D];
    {
      const size_t pz = (size_t)z * plane;
#pragma unroll
      for (int r = 0; r < R + 2; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) pc[r][c] = P[c * N + pz + rowo[r]];
    }
    T zprev[R][NZ];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < NZ; ++c) zprev[r][c] = T(0);
    T part = T(0);
    for (int k = 0; k <= planes; ++k) {  // k = 0: halo plane z0 - 1
      const int zn = z + 1 == nz ? 0 : z + 1;
      const size_t pz = (size_t)z * plane, pzn = (size_t)zn * plane;
      // this plane's material and the next plane's direction
      T pn[R + 2][D], g[R + 1];
      bool sol[R + 1], mk[R + 1];
#pragma unroll
      for (int r = 0; r < R + 2; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) pn[r][c] = P[c * N + pzn + rowo[r]];
#pragma unroll
      for (int r = 0; r < R + 1; ++r) {
        sol[r] = ph[pz + rowo[r]] != 0;
        g[r] = matg ? matg[pz + rowo[r]] : T(0);
        mk[r] = (msk && r >= 1) ? msk[pz + rowo[r]] != 0 : false;
      }
      const bool inner = k >= 1;
      T yp0 = T(0), yp1 = T(0), yp2 = T(0);  // row above: (sxy, syy, syz) or Jy
#pragma unroll
      for (int r = 0; r < R + 1; ++r) {
        const bool out = inner && own && r >= 1 && r <= wy;
        T pr[D];
#pragma unroll
        for (int c = 0; c < D; ++c) pr[c] = __shfl_down_sync(FULL, pc[r][c], 1);
        if constexpr (D == 3) {
          const T ux = pc[r][0], uy = pc[r][1], uz = pc[r][2];
          const T exx = (pr[0] - ux) * ih;
          const T eyy = (pc[r + 1][1] - uy) * ih;
          const T ezz = (pn[r][2] - uz) * ih;
          const T eyz = T(0.5) * ((pn[r][1] - uy) + (pc[r + 1][2] - uz)) * ih;
          const T exz = T(0.5) * ((pn[r][0] - ux) + (pr[2] - uz)) * ih;
          const T exy = T(0.5) * ((pc[r + 1][0] - ux) + (pr[1] - uy)) * ih;
          const T gg = matg ? g[r] : T(1);
          const T lam = gg * (sol[r] ? lam1 : lam0), mu = gg * (sol[r] ? mu1 : mu0);
          const T lt = lam * (exx + eyy + ezz), m2 = T(2) * mu;
          const T sxx = lt + m2 * exx, syy = lt + m2 * eyy, szz = lt + m2 * ezz;
          const T syz = m2 * eyz, sxz = m2 * exz, sxy = m2 * exy;
          const T lxx = __shfl_up_sync(FULL, sxx, 1), lxy = __shfl_up_sync(FULL, sxy, 1),
                  lxz = __shfl_up_sync(FULL, sxz, 1);
          if (out) {
            const size_t gi = pz + rowo[r];
            v.q[gi] = ((lxx - sxx) + (yp0 - sxy) + (zprev[r - 1][0] - sxz)) * ih;
            v.q[N + gi] = ((lxy - sxy) + (yp1 - syy) + (zprev[r - 1][1] - syz)) * ih;
            v.q[2 * N + gi] = ((lxz - sxz) + (yp2 - syz) + (zprev[r - 1][2] - szz)) * ih;
            part += exx * sxx + eyy * syy + ezz * szz + T(2) * (eyz * syz + exz * sxz + exy * sxy);
          }
          if (r >= 1) {
            zprev[r - 1][0] = sxz;
            zprev[r - 1][1] = syz;
            zprev[r - 1][2] = szz;
          }
          yp0 = sxy;
          yp1 = syy;
          yp2 = syz;
        } else {
          const T p = pc[r][0];
          const T kap = sol[r] ? kap1 : kap0;
          const T gx = (pr[0] - p) * ih, gy = (pc[r + 1][0] - p) * ih, gz = (pn[r][0] - p) * ih;
          const T jx = kap * gx, jy = kap * gy, jz = kap * gz;
          const T ljx = __shfl_up_sync(FULL, jx, 1);
          if (out) {
            const size_t gi = pz + rowo[r];
            const T c0 = c0c + g[r];
            T q = c0 * p + ((ljx - jx) + (yp0 - jy) + (zprev[r - 1][0] - jz)) * ih;
            if (mk[r]) q = T(0);
            v.q[gi] = q;
            part += c0 * p * p + kap * (gx * gx + gy * gy + gz * gz);
          }
          if (r >= 1) zprev[r - 1][0] = jz;
          yp0 = jy;
        }
      }
#pragma unroll
      for (int r = 0; r < R + 2; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) pc[r][c] = pn[r][c];
      z = zn;
    }
    acc.add(part);
  }
  double* partials = v.partials + (size_t)bp * gridDim.x;
  if (v.nsten > 0) {  // deferred: the update kernel's blocks sum the partials
    store_deferred_partial<T>(acc, partials + blockIdx.x, redf, red);
    return;
  }
  const double bt[1] = {acc.block_total(redf, red)};
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, int D>
cudaError_t launch_sten2(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  static_assert(kStrip2 == 30 && kSten2Threads == 256, "sten2_blocks assumes 30-column strips, 8 warps");
  const dim3 grid(sten2_blocks(op.nx, op.ny, ss), ss.batch);
  if (ss.ty == 4) return launch_dep(k_sten2<T, D, 4>, grid, dim3(kSten2Threads), 0, st, op, v);
  return launch_dep(k_sten2<T, D, 8>, grid, dim3(kSten2Threads), 0, st, op, v);
}

template <typename T, int D>
cudaError_t launch_sten3(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  const dim3 grid(sten3_blocks(op.nx, op.ny, op.nz, ss), ss.batch);
  if (ss.ty != 4) return cudaErrorInvalidValue;
  return launch_dep(k_sten3<T, D, 4>, grid, dim3(kSten2Threads), 0, st, op, v, ss.zc);
}

}  // namespace fftmech
