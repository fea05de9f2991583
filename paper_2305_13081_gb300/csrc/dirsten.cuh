// Direction and stencil of the split PCG iteration in one kernel (2D grids
// where the iteration is latency-bound): z = x-IFFT(S), p = z + beta p_old,
// then q = K p and the block's share of <p, K p> (stencil.cuh gives the
// operator, Eq. solid with the forward-difference gradient of Sec. 2.6, or
// the scalar c0 + grad+^T kap grad+ of Eqs. diffusion-final and crack-fft).
//
// A block owns the rows y0 .. y0 + nl - 1. The stencil at row y needs the
// direction on rows y - 1 .. y + 1 (the stress at y - 1 and y uses the
// forward difference to the next row), so the block transforms its rows
// and one halo row on either side, nl + 2 rows in all: the direction of a
// halo row is computed again by the block that owns it, with the same
// arithmetic, and the halo rows cost nothing but their transforms. The
// old direction of a halo row must still be the old one when this block
// reads it, so the new direction goes to a second buffer (p_out) and the
// update kernel, which reads it next, copies it back over p_in.
//
// Steps: the scalars (direction_scalars), the spectral rows and the old
// direction of the nl + 2 rows into shared memory, the inverse transforms,
// p on all nl + 2 rows in shared memory (stored for the own rows), the
// stress (flux) on rows y0 - 1 .. y0 + nl - 1 into shared memory over the
// dead spectral rows, then q on the own rows and the energy partial.
// The material of the stress rows (phase, degradation or reaction field)
// and the mask are loaded with all of a thread's loads in flight at once,
// before the reduction, so their latency hides behind it. Shared memory:
// DsLayout.
#pragma once

#include "lines.cuh"

namespace fftmech {

template <typename T, int D, int FX, int NX>
__global__ void FFTMECH_BOUNDS_L k_xds(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int L) {
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const int bp = blockIdx.y;
  line_views<T, D>(op, v, bp, N, (long long)N);
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  grid_dep_sync();  // the plan is constant; everything below follows the previous kernel
  const bool lead = v.ctl.direct && blockIdx.x == 0 && threadIdx.x == 0;
  if (done_flag(v.sc)) {
    if (lead) loop_decide(v.ctl, 0, 0);
    return;
  }
  const DsLayout<T, D> lay(nx, L);
  const int y0 = blockIdx.x * L;
  const int nl = min(L, ny - y0);
  const int W = nl + 2;                                    // rows y0 - 1 .. y0 + nl
  const int ya = y0 == 0 ? ny - 1 : y0 - 1;                // halo row above
  const int yb = y0 + nl == ny ? 0 : y0 + nl;              // halo row below
  cx<T>* F = reinterpret_cast<cx<T>*>(smem + lay.F);
  T* PO = reinterpret_cast<T*>(smem + lay.PO);
  T* MG = reinterpret_cast<T*>(smem + lay.MG);
  uint8_t* PH = smem + lay.PH;
  uint8_t* MK = smem + lay.MK;
  const size_t WS = (size_t)W * nx;  // one component of PO
  const FastDiv dn(nx);
  auto row_of = [&](int i) { return NX > 0 ? i / NX : dn.div(i); };  // local row of local index i
  // rows of the block in shared memory: the halo row above, the own rows,
  // the halo row below (each a contiguous run in global memory)
  auto copy_rows = [&](auto* dst, const auto* src) {
    g2s_async(dst, src + (size_t)ya * nx, nx);
    g2s_async(dst + nx, src + (size_t)y0 * nx, nl * nx);
    g2s_async(dst + (size_t)(nl + 1) * nx, src + (size_t)yb * nx, nx);
  };
  const bool early = v.ncol > 0;  // the copies do not depend on beta: start them before the reduction
  if (early) {
#pragma unroll
    for (int c = 0; c < D; ++c) copy_rows(PO + c * WS, v.p_in + c * N);
    copy_rows(F, v.S);
  }
  // material of the stress rows (local rows 0 .. nl) and the mask of all
  // W rows: eight loads in flight per thread, then the stores
  const T* __restrict__ matg = (D == 2) ? op.g : op.c0f;
  const bool masked = (D == 1) && op.mask;
  {
    const int bd = blockDim.x;
    const int nm = (masked ? W : nl + 1) * nx;
    for (int i0 = threadIdx.x; i0 < nm; i0 += 8 * bd) {
      uint8_t ph8[8], mk8[8];
      T g8[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = i0 + k * bd;
        if (i < nm) {
          const int j = row_of(i), x = i - j * nx;
          const int y = j == 0 ? ya : (j == nl + 1 ? yb : y0 + j - 1);
          const size_t gi = (size_t)y * nx + x;
          if (j <= nl) {
            ph8[k] = op.phase[gi];
            if (matg) g8[k] = matg[gi];
          }
          if (masked) mk8[k] = op.mask[gi];
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = i0 + k * bd;
        if (i < nm) {
          if (i < (nl + 1) * nx) {
            PH[i] = ph8[k];
            if (matg) MG[i] = g8[k];
          }
          if (masked) MK[i] = mk8[k];
        }
      }
    }
  }
  T b;
  if (direction_scalars<T>(v, bp, N, lead, b)) {
    g2s_async_wait();
    return;
  }
  const bool with_old = b != T(0);  // the first iteration has p = z
  if (!early) {
    if (with_old) {
#pragma unroll
      for (int c = 0; c < D; ++c) copy_rows(PO + c * WS, v.p_in + c * N);
    }
    copy_rows(F, v.S);
  }
  g2s_async_wait();
  __syncthreads();
  if constexpr (NX > 0) fftc<T, 1, NX, false>(F, px_s.tw, W);
  else fft_lines<T, 1, FX>(F, px_s, W, nx, 1, false);
  // p on every row; the own rows also to global memory
  const size_t o0 = (size_t)y0 * nx - nx;  // global index of local index i of an own row: o0 + i
  for (int i = threadIdx.x; i < W * nx; i += blockDim.x) {
    T z[D];
    z[0] = F[i].re;
    if constexpr (D == 2) z[1] = F[i].im;
    if (masked && MK[i]) z[0] = T(0);
    const bool own = i >= nx && i < (nl + 1) * nx;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T p = z[c];
      if (with_old) p += b * PO[c * WS + i];
      PO[c * WS + i] = p;
      if (own) v.p_out[c * N + o0 + i] = p;
    }
  }
  __syncthreads();
  // stress (flux) on the local rows 0 .. nl (grid rows y0 - 1 .. y0 + nl - 1)
  // over the dead spectral rows; the energy of the own rows
  T* SG = reinterpret_cast<T*>(F);
  const int SR = (nl + 1) * nx;  // one stress component
  const T ih = op.ih_t;
  const T lam0 = op.lam_t[0], lam1 = op.lam_t[1], mu0 = op.mu_t[0], mu1 = op.mu_t[1];
  const T kap0 = op.kap_t[0], kap1 = op.kap_t[1];
  const T c0c = op.c0c_t;
  Acc<T> acc;
  T part = T(0);
  int cnt = 0;
  for (int i = threadIdx.x; i < SR; i += blockDim.x) {
    const int j = row_of(i), x = i - j * nx;
    const int xp = x + 1 == nx ? 0 : x + 1;
    const bool sol = PH[i] != 0;
    const int ix = j * nx + xp, iy = i + nx;  // right and lower neighbours in PO
    if constexpr (D == 2) {
      const T* P0 = PO;
      const T* P1 = PO + WS;
      const T exx = (P0[ix] - P0[i]) * ih;
      const T eyy = (P1[iy] - P1[i]) * ih;
      const T exy = T(0.5) * ((P0[iy] - P0[i]) + (P1[ix] - P1[i])) * ih;
      const T gg = matg ? MG[i] : T(1);
      const T lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
      const T lt = lam * (exx + eyy);
      const T sxx = lt + T(2) * mu * exx, syy = lt + T(2) * mu * eyy, sxy = T(2) * mu * exy;
      SG[i] = sxx;
      SG[SR + i] = syy;
      SG[2 * SR + i] = sxy;
      if (j > 0) {
        part += exx * sxx + eyy * syy + T(2) * exy * sxy;
        if (++cnt == 16) {  // non-negative terms
          acc.add(part);
          part = T(0);
          cnt = 0;
        }
      }
    } else {
      const T pk = PO[i];
      const T kap = sol ? kap1 : kap0;
      const T gx = (PO[ix] - pk) * ih, gy = (PO[iy] - pk) * ih;
      SG[i] = kap * gx;
      SG[SR + i] = kap * gy;
      if (j > 0) {
        const T c0 = c0c + (matg ? MG[i] : T(0));
        part += c0 * pk * pk + kap * (gx * gx + gy * gy);
        if (++cnt == 16) {
          acc.add(part);
          part = T(0);
          cnt = 0;
        }
      }
    }
  }
  acc.add(part);
  __syncthreads();
  // q on the own rows (local stress rows 1 .. nl; the same index i as in PO)
  for (int i = threadIdx.x + nx; i < SR; i += blockDim.x) {
    const int j = row_of(i), x = i - j * nx;
    const int im = x == 0 ? i + nx - 1 : i - 1;  // left neighbour
    if constexpr (D == 2) {
      const T* Sxx = SG;
      const T* Syy = SG + SR;
      const T* Sxy = SG + 2 * SR;
      v.q[o0 + i] = ((Sxx[im] - Sxx[i]) + (Sxy[i - nx] - Sxy[i])) * ih;
      v.q[N + o0 + i] = ((Sxy[im] - Sxy[i]) + (Syy[i - nx] - Syy[i])) * ih;
    } else {
      const T* Jx = SG;
      const T* Jy = SG + SR;
      const T c0 = c0c + (matg ? MG[i] : T(0));
      T qq = c0 * PO[i] + ((Jx[im] - Jx[i]) + (Jy[i - nx] - Jy[i])) * ih;
      if (masked && MK[i]) qq = T(0);
      v.q[o0 + i] = qq;
    }
  }
  __shared__ double red[32];
  __shared__ float redf[64];
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

template <typename T, int D, int FX, int NX>
cudaError_t launch_xds(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                       cudaStream_t st) {
  const int L = ls.L_ds;
  if (L < 1) return cudaErrorInvalidValue;
  const size_t sm = DsLayout<T, D>(op.nx, L).total + tw_smem_bytes<T>(op.nx);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_xds<T, D, FX, NX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid((op.ny + L - 1) / L, ls.batch);
  return launch_dep(k_xds<T, D, FX, NX>, grid, dim3(ls.thr_ds), sm, st, op, v, px, L);
}

#define FFTMECH_INST_XDS_TD(T, D, F, NX)                                                                   \
  template cudaError_t launch_xds<T, D, F, NX>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&, \
                                               const LineShape&, cudaStream_t);
#define FFTMECH_INST_XDS_T(T, F) \
  FFTMECH_INST_XDS_TD(T, 1, F, 0) \
  FFTMECH_INST_XDS_TD(T, 2, F, 0)
#define FFTMECH_INST_XDS_FIXED(NX)          \
  FFTMECH_INST_XDS_TD(float, 1, FAM_ALL, NX) \
  FFTMECH_INST_XDS_TD(float, 2, FAM_ALL, NX)

}  // namespace fftmech
