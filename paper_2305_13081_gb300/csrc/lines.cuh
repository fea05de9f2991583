// x-line kernels of the split PCG iteration (2D and 3D): the direction
// kernel (z = x-IFFT(S), p = z + beta p_old) and the update kernel
// (u += alpha p, r -= alpha q, S = x-FFT(r)). Neither needs a neighbour
// line, so a block takes L whole lines with no halo and no transform is
// computed twice; the stencil q = K p and <p, K p> run in their own kernel
// (stencil.cuh) between the two.
//
// Spectral rows. DIM = 2: one complex row of nx per x line, the D = 2
// components packed as (r_x + i r_y), a scalar as (r + 0 i). DIM = 3: the
// packed (x, y) pair as nx complex numbers (D = 3) followed by the half
// spectrum (nx/2 + 1 numbers) of the remaining real component (r_z, or the
// scalar for D = 1); a real line's transform is Hermitian, so the other
// half is rebuilt by conjugate symmetry before the inverse transform.
#pragma once

#include <atomic>

#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"
#include "fftc.cuh"

namespace fftmech {

#define FFTMECH_BOUNDS_L __launch_bounds__(512, 2)

template <int DIM, int D>
struct LineLayout {
  // complex fields through the x transform: DIM 2 one packed field; DIM 3
  // the packed pair (D = 3) and the half-spectrum field
  static constexpr int NF = DIM == 2 ? 1 : (D == 3 ? 2 : 1);
  static constexpr bool HALF = DIM == 3;  // last field stored as a half spectrum
};

__host__ __device__ inline int spec_row(int nx, int D, int dim) { return dim == 2 ? nx : nxs_of(nx, D); }

// Problem b of a uniform batch: fields at b N (d-component fields at b D N),
// spectrum at b sst.
template <typename T, int D>
__device__ __forceinline__ void line_views(Op<T>& op, Vec2<T>& v, int b, size_t N, long long sst) {
  const size_t o1 = (size_t)b * N, oD = (size_t)b * D * N;
  op.phase += o1;
  if (op.g) op.g += o1;
  if (op.c0f) op.c0f += o1;
  if (op.mask) op.mask += o1;
  if (v.u) v.u += oD;
  if (v.uh) v.uh += oD;
  if (v.ul) v.ul += oD;
  v.r += oD;
  if (v.p_in) v.p_in += oD;
  if (v.p_out) v.p_out += oD;
  if (v.p_copy) v.p_copy += oD;
  if (v.q) v.q += oD;
  v.S += (size_t)b * sst;
  v.sc += b;
}

// The direction's scalars, for every thread of the block. With a deferred
// reduction of the last column pass (an ITER or TRUE pass, ncol > 0):
// <r, M^-1 r>, convergence and beta in every block; block 0 writes the
// scalars that nothing in the kernel reads (rz_next, rz_true, beta; rz and
// iter only when the problem stops here), the decisions in thread 0 only
// (FP64 runs at a small fraction of FP32). Otherwise the column pass has
// finalised the iteration and beta is read. lead: the thread that takes
// the loop decisions of a one-problem solve. Returns true when the problem
// stops here.
template <typename T>
__device__ __forceinline__ bool direction_scalars(const Vec2<T>& v, int bp, size_t N, bool lead, T& b) {
  if (v.ncol > 0) {
    // deferred reduction of the last column pass (an ITER or TRUE pass):
    // <r, M^-1 r>, convergence and beta in every block; block 0 writes the
    // scalars that nothing in this kernel reads (rz_next, rz_true, beta; rz
    // and iter only when the problem stops here)
    // (the decisions in thread 0 only: FP64 runs at a small fraction of FP32)
    __shared__ float redfx[64];
    __shared__ double redx[32];
    __shared__ T b_s;
    __shared__ int stop_s;
    SolverScalars* s = v.sc;
    const double tsum = deferred_total<T>(v.pcol + (size_t)bp * v.ncol, v.ncol, redfx, redx);
    if (threadIdx.x == 0) {
      const bool w0 = blockIdx.x == 0;
      const double tot = tsum * (1.0 / (double)N);
      const int is_true = vol_readi(&s->col_true);
      stop_s = 1;
      if (!isfinite(tot)) {
        if (w0) {
          s->rz = tot;
          s->done = 1;
          s->status = FFTMECH_ERR_NONFINITE;
          if (v.mode) v.mode[bp] = 0;
        }
      } else if (tot <= s->tol2 * s->rz0 || vol_readi(&s->iter) + 1 >= s->max_iter) {
        // converged, or the iteration limit reached with this column pass
        if (w0) {
          const bool ok = tot <= s->tol2 * s->rz0;
          s->iter += 1;
          if (is_true) s->rz_true = tot;
          s->rz = tot;
          s->done = 1;
          s->status = ok ? FFTMECH_OK : FFTMECH_ERR_NOT_CONVERGED;
          if (v.mode) v.mode[bp] = 0;
        }
      } else {
        double beta = tot / vol_read(&s->rz);
        // a replaced residual larger than the recursive one it replaces means
        // the float recursion had drifted: restart the direction instead
        if (is_true && beta > 1.0) beta = 0.0;
        if (w0) {
          // rz_next is committed to rz by block 0 of a later kernel
          s->rz_next = tot;
          s->rz_pending = 1;
          if (is_true) s->rz_true = tot;
          set_beta(s, beta);
          const int next = reliable_next(s, tot, is_true, vol_readi(&s->iter) + 1);
          if (v.mode) v.mode[bp] = next;
          if (lead) loop_decide(v.ctl, 1, next);
        }
        b_s = (T)beta;
        stop_s = 0;
      }
      if (lead && stop_s) loop_decide(v.ctl, 0, 0);
    }
    __syncthreads();
    if (stop_s) return true;
    b = b_s;
  } else {
    // the column pass finalised the iteration (and chose the next mode)
    if (lead) loop_decide(v.ctl, 1, v.mode ? vol_readi(v.mode + bp) == 1 : 0);
    if constexpr (sizeof(T) == 4) b = vol_readf(&v.sc->beta_f);
    else b = vol_read(&v.sc->beta);
  }
  return false;
}

// ---------------------------------------------------------------- direction
// Lines l0 .. l0 + L - 1 (flattened (z, y) index): z = x-IFFT(S), masked
// voxels (D = 1) 0, p = z + beta p_old. Shared memory: [twiddles]
// [F: NF L complex lines] [PO: old direction, D L lines] [MK: L nx mask bytes].
template <typename T, int D, int FX, int DIM, int NX>
__global__ void FFTMECH_BOUNDS_L k_xdir(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int L, long long sst) {
  using LL = LineLayout<DIM, D>;
  const int nx = op.nx;
  const int nlines = op.ny * op.nz;
  const size_t N = (size_t)nx * nlines;
  const int bp = blockIdx.y;
  line_views<T, D>(op, v, bp, N, sst);
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  grid_dep_sync();  // the plan is constant; everything below follows the previous kernel
  // loop decisions of a one-problem solve are taken here, by block 0's thread 0
  const bool lead = v.ctl.direct && blockIdx.x == 0 && threadIdx.x == 0;
  if (done_flag(v.sc)) {
    if (lead) loop_decide(v.ctl, 0, 0);
    return;
  }
  const int l0 = blockIdx.x * L;
  const int nl = min(L, nlines - l0);
  const int nxs = spec_row(nx, D, DIM);
  const int nxa = (DIM == 3 && D == 3) ? nx : 0;  // packed field's length in a 3D row
  const int nxh = nx / 2 + 1;
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  cx<T>* FB = F + (size_t)(LL::NF - 1) * nl * nx;  // the half-spectrum field's lines (DIM 3)
  T* PO = reinterpret_cast<T*>(smem + align16((size_t)LL::NF * L * nx * sizeof(cx<T>)));
  const size_t t0 = (size_t)l0 * nx;
  // 2D with a deferred reduction: the copies of the spectral rows and the
  // old direction do not depend on beta, so they start before the reduction
  const bool early = DIM == 2 && v.ncol > 0;
  if (early) {
#pragma unroll
    for (int c = 0; c < D; ++c) g2s_async(PO + (size_t)c * nl * nx, v.p_in + c * N + t0, nl * nx);
    g2s_async(F, v.S + t0, nl * nx);
  }
  T b;
  if (direction_scalars<T>(v, bp, N, lead, b)) {
    g2s_async_wait();
    return;
  }
  const bool with_old = b != T(0);  // the first iteration has p = z
  // the old direction and the 2D spectral rows by asynchronous copies (unless
  // already started); the mask and the 3D spectral rows by loads in flight
  // meanwhile; one wait
  if (with_old && !early) {
#pragma unroll
    for (int c = 0; c < D; ++c) g2s_async(PO + (size_t)c * nl * nx, v.p_in + c * N + t0, nl * nx);
  }
  if constexpr (DIM == 2) {
    if (!early) g2s_async(F, v.S + t0, nl * nx);
  } else {
    // the block's spectral rows are one contiguous run of nl nxs numbers:
    // one flattened loop keeps eight loads in flight per thread
    const cx<T>* Sb = v.S + (size_t)l0 * nxs;
    const int ne = nl * nxs;
    const FastDiv dns(nxs);
    const int bd = blockDim.x;
    for (int i = threadIdx.x; i < ne; i += 8 * bd) {
      cx<T> t[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i + k * bd < ne) t[k] = Sb[i + k * bd];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int e = i + k * bd;
        if (e < ne) {
          const int l = dns.div(e), c = e - l * nxs;
          if (c < nxa) F[(size_t)l * nx + c] = t[k];
          else FB[(size_t)l * nx + (c - nxa)] = t[k];
        }
      }
    }
  }
  if (D == 1 && op.mask)
    g2s_vec<8, true>(reinterpret_cast<uint8_t*>(PO) + align16((size_t)D * L * nx * sizeof(T)), op.mask + t0, nl * nx);
  g2s_async_wait();
  __syncthreads();
  if constexpr (LL::HALF) {
    const int nup = nx - nxh;
    const FastDiv dup(nup);
    for (int i = threadIdx.x; i < nl * nup; i += blockDim.x) {
      const int l = dup.div(i), k = nxh + (i - l * nup);
      const cx<T> w = FB[(size_t)l * nx + (nx - k)];
      FB[(size_t)l * nx + k] = mk(w.re, -w.im);
    }
    __syncthreads();
  }
  if constexpr (NX > 0) fftc<T, 1, NX, false>(F, px_s.tw, LL::NF * nl);
  else fft_lines<T, 1, FX>(F, px_s, LL::NF * nl, nx, 1, false);
  const bool masked = (D == 1) && op.mask;
  const uint8_t* MK = reinterpret_cast<const uint8_t*>(PO) + align16((size_t)D * L * nx * sizeof(T));
  for (int i = threadIdx.x; i < nl * nx; i += blockDim.x) {
    T z[D];
    if constexpr (DIM == 2) {
      z[0] = F[i].re;
      if constexpr (D == 2) z[1] = F[i].im;
    } else {
      if constexpr (D == 3) {
        z[0] = F[i].re;
        z[1] = F[i].im;
        z[2] = FB[i].re;
      } else {
        z[0] = FB[i].re;
      }
    }
    if (masked && MK[i]) z[0] = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T p = z[c];
      if (with_old) p += b * PO[(size_t)c * nl * nx + i];
      v.p_out[c * N + t0 + i] = p;
    }
  }
}

// ---------------------------------------------------------------- update
// u += alpha p (double or double-float iterate), r -= alpha q, S = x-FFT(r)
// on lines l0 .. l0 + L - 1. Reliable-update iterations (mode 1) move the
// iterate only. Shared memory: [twiddles] [F: NF L complex lines].
template <typename T, int D, int FX, int DIM, int NX>
__global__ void FFTMECH_BOUNDS_L k_xupd(Op<T> op, Vec2<T> v, FftPlanDev<T> px, int L, long long sst) {
  using LL = LineLayout<DIM, D>;
  const int nx = NX > 0 ? NX : op.nx;  // a constant with a compile-time plan
  const int nlines = op.ny * op.nz;
  const size_t N = (size_t)nx * nlines;
  const int bp = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(px.n);
  const FftPlanDev<T> px_s = plan_to_smem(px, reinterpret_cast<cx<T>*>(smem_all));
  grid_dep_sync();  // the plan is constant; everything below follows the previous kernel
  const int u_only = v.mode ? (v.mode[bp] == 1) : 0;
  line_views<T, D>(op, v, bp, N, sst);
  if (done_flag(v.sc)) return;
  double alpha = 0.0;
  float ah = 0.f, al = 0.f;
  if (v.nsten > 0) {
    // deferred reduction: <p, K p> from the stencil's partials, alpha =
    // <r, M^-1 r> / <p, K p> in every block; block 0 writes the scalars
    // (the decisions in thread 0 only: FP64 runs at a small fraction of FP32)
    __shared__ float redfx[64];
    __shared__ double redx[32];
    __shared__ double a_s;
    __shared__ float ah_s, al_s;
    __shared__ int stop_s;
    const double pq = deferred_total<T>(v.partials + (size_t)bp * v.nsten, v.nsten, redfx, redx);
    if (threadIdx.x == 0) {
      SolverScalars* s = v.sc;
      const bool w0 = blockIdx.x == 0;
      // the residual norm of the last direction: committed by a split
      // stencil kernel, else pending (block 0 commits it here)
      const double rz = rz_current(s);
      if (w0) commit_pending_rz(s);
      stop_s = !(pq > 0.0) || !isfinite(pq);
      if (stop_s) {
        if (w0) {
          s->pq = pq;
          s->done = 1;
          s->status = FFTMECH_ERR_NONFINITE;
        }
      } else {
        const double a0 = rz / pq;
        const float h = (float)a0;
        a_s = a0;
        ah_s = h;
        al_s = (float)(a0 - (double)h);
        if (w0) {
          s->pq = pq;
          s->alpha = a0;
          s->alpha_h = ah_s;
          s->alpha_l = al_s;
        }
      }
    }
    __syncthreads();
    if (stop_s) return;
    if constexpr (sizeof(T) == 4) {
      ah = ah_s;
      al = al_s;
    } else {
      alpha = a_s;
    }
  } else if constexpr (sizeof(T) == 4) {
    ah = vol_readf(&v.sc->alpha_h);
    al = vol_readf(&v.sc->alpha_l);
  } else {
    alpha = vol_read(&v.sc->alpha);
  }
  const T a = sizeof(T) == 4 ? (T)ah : (T)alpha;
  const int l0 = blockIdx.x * L;
  const int nl = min(L, nlines - l0);
  const size_t t0 = (size_t)l0 * nx;
  const int n = nl * nx;
  const int tid = threadIdx.x, bd = blockDim.x;
  cx<T>* F = reinterpret_cast<cx<T>*>(smem);
  cx<T>* FB = F + (size_t)(LL::NF - 1) * nl * nx;
  // iterate update (every mode), residual update and packing (not in a
  // reliable-update iteration) in one pass: all global loads of U voxels are
  // issued before any of their stores. Three components at once would keep
  // fifteen 64-bit addresses live: D = 3 takes one component per pass.
  if constexpr (D == 3) {
    constexpr int U3 = 4;
#pragma unroll 1
    for (int c = 0; c < D; ++c) {
      const size_t gc = (size_t)c * N + t0;
      for (int i0 = tid; i0 < n; i0 += U3 * bd) {
        T p[U3], r[U3], q[U3];
        float uh[U3], ul[U3];
        double ud[U3];
#pragma unroll
        for (int u = 0; u < U3; ++u) {
          const int i = i0 + u * bd;
          if (i < n) {
            p[u] = v.p_in[gc + i];
            if constexpr (sizeof(T) == 4) {
              uh[u] = v.uh[gc + i];
              ul[u] = v.ul[gc + i];
            } else {
              ud[u] = v.u[gc + i];
            }
            if (!u_only) {
              r[u] = v.r[gc + i];
              q[u] = v.q[gc + i];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U3; ++u) {
          const int i = i0 + u * bd;
          if (i < n) {
            if constexpr (sizeof(T) == 4) {
              df_axpy(uh[u], ul[u], ah, al, (float)p[u]);
              v.uh[gc + i] = uh[u];
              v.ul[gc + i] = ul[u];
            } else {
              v.u[gc + i] = ud[u] + alpha * (double)p[u];
            }
            if (!u_only) {
              r[u] -= a * q[u];
              v.r[gc + i] = r[u];
              // packed pair (x, y) in F, z in the half-spectrum field FB
              if (c == 0) F[i].re = r[u];
              else if (c == 1) F[i].im = r[u];
              else FB[i] = mk(r[u], T(0));
            }
          }
        }
      }
    }
  } else {
    constexpr int U = sizeof(T) == 4 ? (D == 1 ? 6 : 3) : (D == 1 ? 4 : 2);
    for (int i0 = tid; i0 < n; i0 += U * bd) {
      T p[U][D], r[U][D], q[U][D];
      float uh[U][D], ul[U][D];
      double ud[U][D];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * bd;
        if (i < n) {
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const size_t g = (size_t)c * N + t0 + i;
            p[u][c] = v.p_in[g];
            if constexpr (sizeof(T) == 4) {
              uh[u][c] = v.uh[g];
              ul[u][c] = v.ul[g];
            } else {
              ud[u][c] = v.u[g];
            }
            if (!u_only) {
              r[u][c] = v.r[g];
              q[u][c] = v.q[g];
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * bd;
        if (i < n) {
#pragma unroll
          for (int c = 0; c < D; ++c) {
            const size_t g = (size_t)c * N + t0 + i;
            if constexpr (sizeof(T) == 4) {
              df_axpy(uh[u][c], ul[u][c], ah, al, (float)p[u][c]);
              v.uh[g] = uh[u][c];
              v.ul[g] = ul[u][c];
            } else {
              v.u[g] = ud[u][c] + alpha * (double)p[u][c];
            }
            if (v.p_copy) v.p_copy[g] = p[u][c];
            if (!u_only) {
              r[u][c] -= a * q[u][c];
              v.r[g] = r[u][c];
            }
          }
          if (!u_only) {
            if constexpr (DIM == 2) F[i] = mk(r[u][0], D == 2 ? r[u][D - 1] : T(0));
            else FB[i] = mk(r[u][0], T(0));
          }
        }
      }
    }
  }
  if (u_only) return;
  __syncthreads();
  if constexpr (NX > 0) fftc<T, -1, NX, false>(F, px_s.tw, LL::NF * nl);
  else fft_lines<T, -1, FX>(F, px_s, LL::NF * nl, nx, 1, false);
  if constexpr (DIM == 2) {
    s2g(v.S + t0, F, n);
  } else {
    const int nxs = spec_row(nx, D, DIM);
    const int nxa = D == 3 ? nx : 0;
    cx<T>* Srow = v.S + (size_t)l0 * nxs;
    const FastDiv dns(nxs);
    for (int i = tid; i < nl * nxs; i += bd) {
      const int l = NX > 0 ? i / nxs : dns.div(i), k = i - l * nxs;
      Srow[i] = k < nxa ? F[(size_t)l * nx + k] : FB[(size_t)l * nx + (k - nxa)];
    }
  }
}

// ---------------------------------------------------------------- launchers

template <typename T, int D, int FX, int DIM, int NX>
cudaError_t launch_xdir(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                        cudaStream_t st) {
  const int L = ls.L_dir;
  const size_t sm = xdir_smem<T>(op.nx, L, D, DIM);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_xdir<T, D, FX, DIM, NX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const int nlines = op.ny * op.nz;
  const dim3 grid((nlines + L - 1) / L, ls.batch);
  return launch_dep(k_xdir<T, D, FX, DIM, NX>, grid, dim3(ls.thr_dir), sm, st, op, v, px, L, ls.sst);
}

template <typename T, int D, int FX, int DIM, int NX>
cudaError_t launch_xupd(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                        cudaStream_t st) {
  const int L = ls.L_upd;
  const size_t sm = xupd_smem<T>(op.nx, L, D, DIM);
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k_xupd<T, D, FX, DIM, NX>, sm, cfg);
  if (e != cudaSuccess) return e;
  const int nlines = op.ny * op.nz;
  const dim3 grid((nlines + L - 1) / L, ls.batch);
  return launch_dep(k_xupd<T, D, FX, DIM, NX>, grid, dim3(ls.thr_upd), sm, st, op, v, px, L, ls.sst);
}

#define FFTMECH_INST_LINES_TD(T, D, F, DIM, NX)                                                                 \
  template cudaError_t launch_xdir<T, D, F, DIM, NX>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&,      \
                                                     const LineShape&, cudaStream_t);                         \
  template cudaError_t launch_xupd<T, D, F, DIM, NX>(const Op<T>&, const Vec2<T>&, const FftPlanDev<T>&,      \
                                                     const LineShape&, cudaStream_t);
#define FFTMECH_INST_LINES_T(T, F)         \
  FFTMECH_INST_LINES_TD(T, 1, F, 2, 0)     \
  FFTMECH_INST_LINES_TD(T, 2, F, 2, 0)     \
  FFTMECH_INST_LINES_TD(T, 1, F, 3, 0)     \
  FFTMECH_INST_LINES_TD(T, 3, F, 3, 0)
// x lines of a compile-time length (float): FX unused
#define FFTMECH_INST_LINES_FIXED(NX)                  \
  FFTMECH_INST_LINES_TD(float, 1, FAM_ALL, 2, NX)     \
  FFTMECH_INST_LINES_TD(float, 2, FAM_ALL, 2, NX)     \
  FFTMECH_INST_LINES_TD(float, 1, FAM_ALL, 3, NX)     \
  FFTMECH_INST_LINES_TD(float, 3, FAM_ALL, 3, NX)

}  // namespace fftmech
