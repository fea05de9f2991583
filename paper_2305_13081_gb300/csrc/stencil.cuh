// Stencil kernels of the split PCG iteration: q = K p and the energy form
// <p, K p> = sum over voxels of eps(p) : g C : eps(p) (elasticity) or
// c0 p^2 + kap |grad+ p|^2 (scalar problems), whose last block sets
// alpha = <r, M^-1 r> / <p, K p>. K = grad+^T [g C sym grad+] (Eq. solid
// with the forward-difference gradient of Sec. 2.6) or c0 + grad+^T kap
// grad+ (Eqs. diffusion-final, crack-fft); masked voxels (Dirichlet) get
// q = 0. Tiles of TX x TY voxels with a one-voxel halo in shared memory;
// 3D tiles march through Zc planes keeping two planes of the direction and
// of the z-differenced stress (or flux) components.
#pragma once

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

// ---------------------------------------------------------------- 2D
// Shared memory: [P: D (TY+2)(TX+2)] [SG: 3 (TY+1)(TX+1)] [MG: (TY+1)(TX+1)]
// [PH: (TY+1)(TX+1) bytes]; P covers x0-1 .. x0+TX, y0-1 .. y0+TY.
template <typename T, int D>
__global__ void FFTMECH_BOUNDS_S k_sten2(Op<T> op, Vec2<T> v, int TX, int TY) {
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  sten_views<T, D>(op, v, bp, N);
  if (done_flag(v.sc)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ float redf[64];
  const int ntx = (nx + TX - 1) / TX;
  const int ty = blockIdx.x / ntx, tx = blockIdx.x - ty * ntx;
  const int x0 = tx * TX, y0 = ty * TY;
  const int wx = min(TX, nx - x0), wy = min(TY, ny - y0);
  const int PW = wx + 2, PHt = wy + 2;  // halo tile of the direction
  const int SW = wx + 1, SH = wy + 1;   // stress / flux positions
  T* P = reinterpret_cast<T*>(smem);
  T* SG = P + (size_t)D * (TY + 2) * (TX + 2);
  T* MG = SG + (size_t)3 * (TY + 1) * (TX + 1);
  uint8_t* PH = reinterpret_cast<uint8_t*>(MG + (size_t)(TY + 1) * (TX + 1));
  const T* matg = (D == 2) ? op.g : op.c0f;
  const int tid = threadIdx.x, bd = blockDim.x;
  {
    const FastDiv dw(PW);
    for (int i = tid; i < PHt * PW; i += bd) {
      const int yy = dw.div(i), xx = i - yy * PW;
      const size_t gi = (size_t)wrapi(y0 - 1 + yy, ny) * nx + wrapi(x0 - 1 + xx, nx);
#pragma unroll
      for (int c = 0; c < D; ++c) P[(size_t)c * PHt * PW + i] = v.p_in[c * N + gi];
    }
    const FastDiv ds(SW);
    for (int i = tid; i < SH * SW; i += bd) {
      const int yy = ds.div(i), xx = i - yy * SW;
      const size_t gi = (size_t)wrapi(y0 - 1 + yy, ny) * nx + wrapi(x0 - 1 + xx, nx);
      if (matg) MG[i] = matg[gi];
      PH[i] = op.phase[gi];
    }
  }
  __syncthreads();
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  const size_t SS = (size_t)SH * SW;
  T part = T(0);
  {
    const FastDiv ds(SW);
    for (int i = tid; i < SH * SW; i += bd) {
      const int yy = ds.div(i), xx = i - yy * SW;
      const int c = yy * PW + xx;  // this position in P
      const bool sol = PH[i] != 0;
      const bool inner = xx >= 1 && yy >= 1;
      if constexpr (D == 2) {
        const T* Ux = P;
        const T* Uy = P + (size_t)PHt * PW;
        const T exx = (Ux[c + 1] - Ux[c]) * ih;
        const T eyy = (Uy[c + PW] - Uy[c]) * ih;
        const T exy = T(0.5) * ((Ux[c + PW] - Ux[c]) + (Uy[c + 1] - Uy[c])) * ih;
        const T gg = matg ? MG[i] : T(1);
        const T lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
        const T lt = lam * (exx + eyy);
        const T sxx = lt + T(2) * mu * exx, syy = lt + T(2) * mu * eyy, sxy = T(2) * mu * exy;
        SG[i] = sxx;
        SG[SS + i] = syy;
        SG[2 * SS + i] = sxy;
        if (inner) part += exx * sxx + eyy * syy + T(2) * exy * sxy;
      } else {
        const T p = P[c];
        const T kap = sol ? kap1 : kap0;
        const T gx = (P[c + 1] - p) * ih, gy = (P[c + PW] - p) * ih;
        SG[i] = kap * gx;
        SG[SS + i] = kap * gy;
        if (inner) part += (c0c + (matg ? MG[i] : T(0))) * p * p + kap * (gx * gx + gy * gy);
      }
    }
  }
  __syncthreads();
  {
    const bool masked = (D == 1) && op.mask;
    const FastDiv dx(wx);
    for (int i = tid; i < wy * wx; i += bd) {
      const int yr = dx.div(i), xr = i - yr * wx;
      const int s = (yr + 1) * SW + (xr + 1);  // position in SG
      const size_t gi = (size_t)(y0 + yr) * nx + x0 + xr;
      if constexpr (D == 2) {
        const T* Sxx = SG;
        const T* Syy = SG + SS;
        const T* Sxy = SG + 2 * SS;
        v.q[gi] = ((Sxx[s - 1] - Sxx[s]) + (Sxy[s - SW] - Sxy[s])) * ih;
        v.q[N + gi] = ((Sxy[s - 1] - Sxy[s]) + (Syy[s - SW] - Syy[s])) * ih;
      } else {
        const T* Jx = SG;
        const T* Jy = SG + SS;
        const T p = P[(yr + 1) * PW + xr + 1];
        T q = (c0c + (matg ? MG[s] : T(0))) * p + ((Jx[s - 1] - Jx[s]) + (Jy[s - SW] - Jy[s])) * ih;
        if (masked && op.mask[gi]) q = T(0);
        v.q[gi] = q;
      }
    }
  }
  Acc<T> acc;
  acc.add(part);
  const double bt[1] = {acc.block_total(redf, red)};
  double* partials = v.partials + (size_t)bp * gridDim.x;
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- 3D
// Direction of plane z (periodic) into ring slot s: the tile with its halo.
template <typename T, int D>
__device__ __forceinline__ void sten3_load_plane(T* P, const T* __restrict__ p, int z, int s, int x0, int y0, int PW,
                                                 int PHt, size_t PS, int nx, int ny, int nz, size_t N,
                                                 const FastDiv& dpw) {
  const size_t pz = (size_t)wrapi(z, nz) * nx * ny;
  T* dst = P + (size_t)s * D * PS;
  for (int i = threadIdx.x; i < PHt * PW; i += blockDim.x) {
    const int yy = dpw.div(i), xx = i - yy * PW;
    const size_t gi = pz + (size_t)wrapi(y0 - 1 + yy, ny) * nx + wrapi(x0 - 1 + xx, nx);
#pragma unroll
    for (int c = 0; c < D; ++c) dst[c * PS + i] = p[c * N + gi];
  }
}

// Shared memory: [P: 2 planes x D (TY+2)(TX+2)] [SP: NP (TY+1)(TX+1)]
// [SZ: 2 planes x NZ (TY+1)(TX+1)] [MG: (TY+1)(TX+1)] [PH: bytes]; NP
// in-plane components (sxx, syy, sxy or Jx, Jy), NZ z-differenced ones
// (sxz, syz, szz or Jz).
template <typename T, int D>
__global__ void FFTMECH_BOUNDS_S k_sten3(Op<T> op, Vec2<T> v, int TX, int TY, int Zc) {
  constexpr int NP = D == 3 ? 3 : 2, NZ = D == 3 ? 3 : 1;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int bp = blockIdx.y;
  sten_views<T, D>(op, v, bp, N);
  if (done_flag(v.sc)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ float redf[64];
  const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty;
  const int tz = t / nty;
  const int x0 = tx * TX, y0 = ty * TY, z0 = tz * Zc;
  const int wx = min(TX, nx - x0), wy = min(TY, ny - y0), planes = min(Zc, nz - z0);
  const int PW = wx + 2, PHt = wy + 2;
  const int SW = wx + 1, SH = wy + 1;
  const size_t PS = (size_t)(TY + 2) * (TX + 2);  // one component of one P plane
  const size_t SS = (size_t)(TY + 1) * (TX + 1);  // one stress component
  T* P = reinterpret_cast<T*>(smem);
  T* SP = P + 2 * D * PS;
  T* SZ = SP + NP * SS;
  T* MG = SZ + 2 * NZ * SS;
  uint8_t* PH = reinterpret_cast<uint8_t*>(MG + SS);
  const T* matg = (D == 3) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  const int tid = threadIdx.x, bd = blockDim.x;
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  const FastDiv dpw(PW), dsw(SW), dwx(wx);
  T part = T(0);
  sten3_load_plane<T, D>(P, v.p_in, z0 - 1, 0, x0, y0, PW, PHt, PS, nx, ny, nz, N, dpw);
  for (int zz = z0 - 1; zz < z0 + planes; ++zz) {
    const int cur = (zz - z0 + 1) & 1, nxt = cur ^ 1;
    const bool inner_plane = zz >= z0;
    const size_t pz = (size_t)wrapi(zz, nz) * plane;
    sten3_load_plane<T, D>(P, v.p_in, zz + 1, nxt, x0, y0, PW, PHt, PS, nx, ny, nz, N, dpw);
    for (int i = tid; i < SH * SW; i += bd) {
      const int yy = dsw.div(i), xx = i - yy * SW;
      const size_t gi = pz + (size_t)wrapi(y0 - 1 + yy, ny) * nx + wrapi(x0 - 1 + xx, nx);
      if (matg) MG[i] = matg[gi];
      PH[i] = op.phase[gi];
    }
    __syncthreads();
    const T* Pc = P + (size_t)cur * D * PS;
    const T* Pn = P + (size_t)nxt * D * PS;
    T* Zc_ = SZ + (size_t)cur * NZ * SS;
    const T* Zp = SZ + (size_t)nxt * NZ * SS;  // previous plane
    for (int i = tid; i < SH * SW; i += bd) {
      const int yy = dsw.div(i), xx = i - yy * SW;
      const int c = yy * PW + xx;
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
    __syncthreads();
    if (inner_plane) {
      for (int i = tid; i < wy * wx; i += bd) {
        const int yr = dwx.div(i), xr = i - yr * wx;
        const int s = (yr + 1) * SW + (xr + 1);
        const size_t gi = pz + (size_t)(y0 + yr) * nx + x0 + xr;
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
          const T p = Pc[(yr + 1) * PW + xr + 1];
          T q = (c0c + (matg ? MG[s] : T(0))) * p +
                ((Jx[s - 1] - Jx[s]) + (Jy[s - SW] - Jy[s]) + (Zp[s] - Zc_[s])) * ih;
          if (masked && op.mask[gi]) q = T(0);
          v.q[gi] = q;
        }
      }
    }
    __syncthreads();
  }
  Acc<T> acc;
  acc.add(part);
  const double bt[1] = {acc.block_total(redf, red)};
  double* partials = v.partials + (size_t)bp * gridDim.x;
  if (publish_partials<1>(bt, partials, &v.sc->cnt[0])) {
    double tot[1];
    gather_partials<1>(tot, partials, &v.sc->cnt[0], red);
    if (threadIdx.x == 0) finalize_direction(v.sc, tot[0]);
  }
}

// ---------------------------------------------------------------- launchers
template <typename K>
static cudaError_t set_smem_s(K kernel, size_t bytes, int& configured) {
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

template <typename T, int D>
cudaError_t launch_sten2(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  const size_t sm = sten2_smem<T>(ss.tx, ss.ty, D);
  static int cfg = 0;
  cudaError_t e = set_smem_s(k_sten2<T, D>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.nx + ss.tx - 1) / ss.tx) * ((op.ny + ss.ty - 1) / ss.ty), ss.batch);
  k_sten2<T, D><<<grid, ss.threads, sm, st>>>(op, v, ss.tx, ss.ty);
  return cudaGetLastError();
}

template <typename T, int D>
cudaError_t launch_sten3(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st) {
  const size_t sm = sten3_smem<T>(ss.tx, ss.ty, D);
  static int cfg = 0;
  cudaError_t e = set_smem_s(k_sten3<T, D>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(((op.nx + ss.tx - 1) / ss.tx) * ((op.ny + ss.ty - 1) / ss.ty) * ((op.nz + ss.zc - 1) / ss.zc),
                  ss.batch);
  k_sten3<T, D><<<grid, ss.threads, sm, st>>>(op, v, ss.tx, ss.ty, ss.zc);
  return cudaGetLastError();
}

}  // namespace fftmech
