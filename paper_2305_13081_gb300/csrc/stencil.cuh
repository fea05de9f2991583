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

#include <atomic>

#include <algorithm>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

#define FFTMECH_BOUNDS_S __launch_bounds__(256)

static __device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

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

// Wrap an index at most one period outside [0, n).
static __device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

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
// Shared memory: [P: 2 planes x D (TY+2)(TX+2)] [SP: NP (TY+1)(TX+1)]
// [SZ: 2 planes x NZ (TY+1)(TX+1)] [MG: (TY+1)(TX+1)] [PH: bytes]; NP
// in-plane components (sxx, syy, sxy or Jx, Jy), NZ z-differenced ones
// (sxz, syz, szz or Jz). blockDim = (TX, TY): thread (tx, ty) owns tile
// column tx (and the halo columns TX, TX + 1 when tx < 2) and tile row ty.
template <typename T, int D, int TX, int TY>
__global__ void FFTMECH_BOUNDS_S k_sten3(Op<T> op, Vec2<T> v, int Zc) {
  constexpr int NP = D == 3 ? 3 : 2, NZ = D == 3 ? 3 : 1;
  constexpr int PW = TX + 2, SW = TX + 1;
  constexpr size_t PS = (size_t)(TY + 2) * PW, SS = (size_t)(TY + 1) * SW;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  sten_views<T, D>(op, v, bp, N);
  grid_dep_sync();
  if (done_flag(v.sc)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ float redf[64];
  T* P = reinterpret_cast<T*>(smem);
  T* SP = P + 2 * D * PS;
  T* SZ = SP + NP * SS;
  T* MG = SZ + 2 * NZ * SS;
  uint8_t* PH = reinterpret_cast<uint8_t*>(MG + SS);
  const T* matg = (D == 3) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  const int tx = threadIdx.x, ty = threadIdx.y, TY4 = blockDim.y;
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
  const int nitems = ntx * nty * ((nz + Zc - 1) / Zc);
  Acc<T> acc;
  // bricks blockIdx.x, blockIdx.x + gridDim.x, ...: one reduction ticket per block
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    T part = T(0);
    int t = item;
    const int txi = t % ntx;
    t /= ntx;
    const int tyi = t % nty;
    const int tzi = t / nty;
    const int x0 = txi * TX, y0 = tyi * TY, z0 = tzi * Zc;
    const int wx = min(TX, nx - x0), wy = min(TY, ny - y0), planes = min(Zc, nz - z0);
    const int xa = wrap1(x0 - 1 + tx, nx);
    const bool ha = tx < wx + 2;
    const bool hb = tx < 2 && TX + tx < wx + 2;
    const int xb = wrap1(x0 - 1 + TX + tx, nx);
    // direction of plane z into ring slot s (tile with halo)
    auto load_p = [&](int z, int slot) {
      const size_t pz = (size_t)wrap1(z, nz) * plane;
      T* dst = P + (size_t)slot * D * PS;
      for (int yy = ty; yy < wy + 2; yy += TY4) {
        const size_t rowg = pz + (size_t)wrap1(y0 - 1 + yy, ny) * nx;
        T va[D], vb[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          va[c] = ha ? v.p_in[c * N + rowg + xa] : T(0);
          vb[c] = hb ? v.p_in[c * N + rowg + xb] : T(0);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
          if (ha) dst[c * PS + yy * PW + tx] = va[c];
          if (hb) dst[c * PS + yy * PW + TX + tx] = vb[c];
        }
      }
    };
    load_p(z0 - 1, 0);
    for (int zz = z0 - 1; zz < z0 + planes; ++zz) {
      const int cur = (zz - z0 + 1) & 1, nxt = cur ^ 1;
      const bool inner_plane = zz >= z0;
      const size_t pz = (size_t)wrap1(zz, nz) * plane;
      load_p(zz + 1, nxt);
      for (int yy = ty; yy <= wy; yy += TY4) {
        const size_t rowg = pz + (size_t)wrap1(y0 - 1 + yy, ny) * nx;
        if (ha && tx <= wx) {
          MG[yy * SW + tx] = matg ? matg[rowg + xa] : T(0);
          PH[yy * SW + tx] = op.phase[rowg + xa];
        }
        if (hb && TX + tx <= wx) {
          MG[yy * SW + TX + tx] = matg ? matg[rowg + xb] : T(0);
          PH[yy * SW + TX + tx] = op.phase[rowg + xb];
        }
      }
      __syncthreads();
      const T* Pc = P + (size_t)cur * D * PS;
      const T* Pn = P + (size_t)nxt * D * PS;
      T* Zc_ = SZ + (size_t)cur * NZ * SS;
      const T* Zp = SZ + (size_t)nxt * NZ * SS;  // previous plane
      for (int yy = ty; yy <= wy; yy += TY4) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int xx = h == 0 ? tx : TX + tx;
          if (xx > wx || (h == 1 && tx >= 1)) continue;
          const int c = yy * PW + xx, i = yy * SW + xx;
          const bool sol = PH[i] != 0;
          const bool inner = inner_plane && xx >= 1 && yy >= 1;
          if constexpr (D == 3) {
            const T* Ux = Pc;
            const T* Uy = Pc + PS;
            const T* Uz = Pc + 2 * PS;
            const T ux = Ux[c], uy = Uy[c], uz = Uz[c];
            const T exx = (Ux[c + 1] - ux) * ih;
            const T eyy = (Uy[c + PW] - uy) * ih;
            const T ezz = (Pn[2 * PS + c] - uz) * ih;
            const T eyz = T(0.5) * ((Pn[PS + c] - uy) + (Uz[c + PW] - uz)) * ih;
            const T exz = T(0.5) * ((Pn[c] - ux) + (Uz[c + 1] - uz)) * ih;
            const T exy = T(0.5) * ((Ux[c + PW] - ux) + (Uy[c + 1] - uy)) * ih;
            const T gg = matg ? MG[i] : T(1);
            const T lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
            const T lt = lam * (exx + eyy + ezz), m2 = T(2) * mu;
            const T sxx = lt + m2 * exx, syy = lt + m2 * eyy, szz = lt + m2 * ezz;
            const T syz = m2 * eyz, sxz = m2 * exz, sxy = m2 * exy;
            SP[i] = sxx;
            SP[SS + i] = syy;
            SP[2 * SS + i] = sxy;
            Zc_[i] = sxz;
            Zc_[SS + i] = syz;
            Zc_[2 * SS + i] = szz;
            if (inner) part += exx * sxx + eyy * syy + ezz * szz + T(2) * (eyz * syz + exz * sxz + exy * sxy);
          } else {
            const T p = Pc[c];
            const T kap = sol ? kap1 : kap0;
            const T gx = (Pc[c + 1] - p) * ih, gy = (Pc[c + PW] - p) * ih, gz = (Pn[c] - p) * ih;
            SP[i] = kap * gx;
            SP[SS + i] = kap * gy;
            Zc_[i] = kap * gz;
            if (inner) part += (c0c + (matg ? MG[i] : T(0))) * p * p + kap * (gx * gx + gy * gy + gz * gz);
          }
        }
      }
      __syncthreads();
      if (inner_plane && tx < wx) {
        for (int yr = ty; yr < wy; yr += TY4) {
          const int s = (yr + 1) * SW + (tx + 1);
          const size_t gi = pz + (size_t)(y0 + yr) * nx + x0 + tx;
          if constexpr (D == 3) {
            const T* Sxx = SP;
            const T* Syy = SP + SS;
            const T* Sxy = SP + 2 * SS;
            const T* Sxz = Zc_;
            const T* Syz = Zc_ + SS;
            const T* Szz = Zc_ + 2 * SS;
            v.q[gi] = ((Sxx[s - 1] - Sxx[s]) + (Sxy[s - SW] - Sxy[s]) + (Zp[s] - Sxz[s])) * ih;
            v.q[N + gi] = ((Sxy[s - 1] - Sxy[s]) + (Syy[s - SW] - Syy[s]) + (Zp[SS + s] - Syz[s])) * ih;
            v.q[2 * N + gi] = ((Sxz[s - 1] - Sxz[s]) + (Syz[s - SW] - Syz[s]) + (Zp[2 * SS + s] - Szz[s])) * ih;
          } else {
            const T* Jx = SP;
            const T* Jy = SP + SS;
            const T p = Pc[(yr + 1) * PW + tx + 1];
            T q = (c0c + (matg ? MG[s] : T(0))) * p +
                  ((Jx[s - 1] - Jx[s]) + (Jy[s - SW] - Jy[s]) + (Zp[s] - Zc_[s])) * ih;
            if (masked && op.mask[gi]) q = T(0);
            v.q[gi] = q;
          }
        }
      }
      __syncthreads();
    }
    acc.add(part);
  }
  const double bt[1] = {acc.block_total(redf, red)};
  double* partials = v.partials + (size_t)bp * gridDim.x;
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0 && threadIdx.y == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- launchers
template <typename K>
static cudaError_t set_smem_s(K kernel, size_t bytes, std::atomic<int>& configured) {
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

// 3D tiles: 32 x 8 voxels per 32 x 8 threads.
constexpr int kSten3TX = 32, kSten3TY = 8;

template <typename T, int D>
cudaError_t launch_sten2(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  static_assert(kStrip2 == 30 && kSten2Threads == 256, "sten2_blocks assumes 30-column strips, 8 warps");
  const dim3 grid(sten2_blocks(op.nx, op.ny, ss), ss.batch);
  if (ss.ty == 4) return launch_dep(k_sten2<T, D, 4>, grid, dim3(kSten2Threads), 0, st, op, v);
  return launch_dep(k_sten2<T, D, 8>, grid, dim3(kSten2Threads), 0, st, op, v);
}

template <typename T, int D>
cudaError_t launch_sten3(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  const size_t sm = sten3_smem<T>(kSten3TX, kSten3TY, D);
  static std::atomic<int> cfg{0};
  cudaError_t e = set_smem_s(k_sten3<T, D, kSten3TX, kSten3TY>, sm, cfg);
  if (e != cudaSuccess) return e;
  const int bricks = ((op.nx + kSten3TX - 1) / kSten3TX) * ((op.ny + kSten3TY - 1) / kSten3TY) *
                     ((op.nz + ss.zc - 1) / ss.zc);
  const dim3 grid(ss.grid > 0 ? std::min(ss.grid, bricks) : bricks, ss.batch);
  return launch_dep(k_sten3<T, D, kSten3TX, kSten3TY>, grid, dim3(kSten3TX, kSten3TY), sm, st, op, v, ss.zc);
}

}  // namespace fftmech
