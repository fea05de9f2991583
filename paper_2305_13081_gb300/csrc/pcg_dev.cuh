// Device-side PCG bookkeeping shared by the 2D and 3D kernels: the
// finalisers that the last block of a reduction runs on the solver scalars.
#pragma once

#include "fftmech_internal.cuh"
#include "fftmech.h"

namespace fftmech {

static __device__ __forceinline__ int wrap_y(int y, int ny) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }

static __device__ __forceinline__ int done_flag(const SolverScalars* sc) {
  return *reinterpret_cast<const volatile int*>(&sc->done);
}

// A stopped problem whose FP64 true residual the gate has not seen yet.
static __device__ __forceinline__ bool unchecked_stop(const SolverScalars* sc) {
  return done_flag(sc) && *reinterpret_cast<const volatile int*>(&sc->checked) == 0;
}

static __device__ __forceinline__ double vol_read(const double* p) {
  return *reinterpret_cast<const volatile double*>(p);
}
static __device__ __forceinline__ float vol_readf(const float* p) {
  return *reinterpret_cast<const volatile float*>(p);
}

// ---------------------------------------------------------------- finalisers
static __device__ void finalize_direction(SolverScalars* sc, double pq) {
  sc->pq = pq;
  if (!(pq > 0.0) || !isfinite(pq)) {
    sc->done = 1;
    sc->status = FFTMECH_ERR_NONFINITE;
    return;
  }
  const double a = sc->rz / pq;
  sc->alpha = a;
  sc->alpha_h = (float)a;
  sc->alpha_l = (float)(a - (double)sc->alpha_h);
}

static __device__ __forceinline__ void set_beta(SolverScalars* sc, double b) {
  sc->beta = b;
  sc->beta_f = (float)b;
}

// Reliable updates (MIXED): the mode of the next iteration of a problem
// that continues. After a replacement its residual norm becomes the new
// reference; otherwise the next iteration replaces the float recursive
// residual by the FP64 true residual once <r, M^-1 r> has fallen 100-fold
// below that reference (the search direction is kept). The test is taken
// only after every kReplacePeriod-th iteration, so that the problems of a
// batch that fall due close together are replaced in the same iteration
// (each replacement iteration ends a round of the device-driven loop, with
// its own launches). Single writer.
constexpr int kReplacePeriod = 16;

static __device__ __forceinline__ int reliable_next(SolverScalars* sc, double tot, int was_replacement,
                                                    int iter_after) {
  if (!sc->reliable) return 0;
  if (was_replacement) {
    sc->rz_rep = tot;
    return 0;
  }
  if (tot < 1e-2 * sc->rz_rep && iter_after % kReplacePeriod == 0) {
    sc->nreplace += 1;
    return 1;
  }
  return 0;
}

// Sets loop flag k to `value` in device memory and, when the solve runs as a
// graph that holds the flag's conditional node, the node's condition.
static __device__ __forceinline__ void set_loop_flag(const LoopCtl& c, int k, int value) {
  if (!c.flags) return;
  c.flags[k] = value;
  if (c.have & (1u << k)) cudaGraphSetConditional((cudaGraphConditionalHandle)c.h[k], (unsigned int)value);
}

// Deferred reductions (2D): the direction kernel leaves the new residual
// norm in rz_next (its blocks all read rz as the previous norm, so none of
// them may overwrite it) and block 0 of a later kernel commits it: the
// stencil kernel after a split direction, the update kernel after the fused
// direction-stencil kernel. The commit stores rz before it clears
// rz_pending (release); a block of the committing kernel reads rz_pending
// first (acquire), so it sees either the pending norm in rz_next or the
// committed rz, which are equal (rz_current).
static __device__ __forceinline__ void commit_pending_rz(SolverScalars* sc) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  if (*reinterpret_cast<volatile int*>(&sc->rz_pending)) {
    *reinterpret_cast<volatile double*>(&sc->rz) = *reinterpret_cast<volatile double*>(&sc->rz_next);
    *reinterpret_cast<volatile int*>(&sc->iter) = *reinterpret_cast<volatile int*>(&sc->iter) + 1;
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(&sc->rz_pending), "r"(0) : "memory");
  }
}
static __device__ __forceinline__ double rz_current(const SolverScalars* sc) {
  int pend;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(pend) : "l"(&sc->rz_pending) : "memory");
  return pend ? *reinterpret_cast<const volatile double*>(&sc->rz_next)
              : *reinterpret_cast<const volatile double*>(&sc->rz);
}

// Loop decisions after a direction (single writer): an active problem runs
// an ordinary iteration next, or a replacement iteration; a stopped one
// ends the loop.
// gate: some problem has stopped and awaits its true-residual check (one
// problem: it has stopped).
static __device__ __forceinline__ void loop_decide(const LoopCtl& c, int active, int replace, int gate) {
  set_loop_flag(c, LF_LOOP, active && !replace);
  set_loop_flag(c, LF_REPLACE, active && replace);
  set_loop_flag(c, LF_GATE, gate);
}
static __device__ __forceinline__ void loop_decide(const LoopCtl& c, int active, int replace) {
  loop_decide(c, active, replace, !active);
}

// pmode: this problem's iteration mode (NULL when there is none); ITER and
// TRUE set it for the next iteration (reliable updates).
static __device__ void finalize_col(SolverScalars* sc, int mode, double tot, int* pmode = nullptr) {
  if (mode == COL_NORM) { sc->rz0 = tot; return; }
  if (mode == COL_PLAIN) return;
  if (mode == COL_TRUENORM) { sc->rz_true = tot; return; }
  if (!isfinite(tot)) {
    sc->rz = tot;
    sc->done = 1;
    sc->status = FFTMECH_ERR_NONFINITE;
    return;
  }
  if (mode == COL_INIT) {
    sc->rz = tot;
    sc->rz_rep = tot;
    set_beta(sc, 0.0);
    sc->iter = 0;
    if (tot <= sc->tol2 * sc->rz0) { sc->done = 1; sc->status = FFTMECH_OK; }
    else if (sc->max_iter <= 0) { sc->done = 1; sc->status = FFTMECH_ERR_NOT_CONVERGED; }
    return;
  }
  if (mode == COL_RESTART) {
    // the true residual replaced r after a recursive convergence: restart
    sc->rz = tot;
    sc->rz_true = tot;
    sc->rz_rep = tot;
    set_beta(sc, 0.0);
    if (tot <= sc->tol2 * sc->rz0) { sc->done = 1; sc->status = FFTMECH_OK; }
    else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = FFTMECH_ERR_NOT_CONVERGED; }
    return;
  }
  sc->iter += 1;
  if (mode == COL_TRUE) sc->rz_true = tot;
  const double rz_old = sc->rz;
  sc->rz = tot;
  const bool conv = tot <= sc->tol2 * sc->rz0;
  if (conv || sc->iter >= sc->max_iter) {
    sc->done = 1;
    sc->status = conv ? FFTMECH_OK : FFTMECH_ERR_NOT_CONVERGED;
    if (pmode) *pmode = 0;
    return;
  }
  double beta = tot / rz_old;
  // a replaced residual larger than the recursive one it replaces means the
  // float recursion had drifted: restart the direction instead of mixing
  if (mode == COL_TRUE && beta > 1.0) beta = 0.0;
  set_beta(sc, beta);
  const int next = reliable_next(sc, tot, mode == COL_TRUE, sc->iter);
  if (pmode) *pmode = next;
}

// Deferred reductions (2D): a producer kernel stores one partial per block
// (store_deferred_partial) and takes no ticket; every block of the consuming
// kernel sums the partials itself (deferred_total), in a fixed order, so that
// all blocks obtain the same total. The kernel boundary orders the partial
// stores before these loads. Float kernels keep both sides in double-float
// arithmetic (a partial is the float pair h, l in the 8-byte slot): GB300
// runs FP64 at a small fraction of FP32, and every block of the consumer
// repeats the sum.
template <typename T>
struct Acc;
template <typename T>
__device__ __forceinline__ void store_deferred_partial(Acc<T>& acc, double* slot, float* redf, double* red);

// Total of n partials, valid in thread 0 of the block. The first
// kDeferredWidth threads take part in a fixed pattern (thread t sums
// partials t, t + W, ... in order; then a shuffle tree in each of the W / 32
// warps; then the warp totals in order), so the total does not depend on the
// block size of the kernel that forms it nor on the unrolling. The block
// needs >= W threads.
constexpr int kDeferredWidth = 128;
template <typename T>
__device__ __forceinline__ double deferred_total(const double* partials, int n, float* redf, double* red) {
  constexpr int W = kDeferredWidth;
  constexpr int UN = 8;  // loads in flight per thread: up to 1024 partials in one round trip
  const int tid = flat_tid(), lane = tid & 31, wid = tid >> 5;
  if constexpr (sizeof(T) == 4) {
    const float2* p2 = reinterpret_cast<const float2*>(partials);
    dfloat s{0.f, 0.f};
    if (tid < W) {
      for (int b0 = tid; b0 < n; b0 += UN * W) {
        float2 x[UN];
#pragma unroll
        for (int j = 0; j < UN; ++j) x[j] = b0 + j * W < n ? __ldcg(p2 + b0 + j * W) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < UN; ++j)
          if (b0 + j * W < n) s = df_add(s, dfloat{x[j].x, x[j].y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const dfloat w{__shfl_down_sync(0xffffffffu, s.h, o), __shfl_down_sync(0xffffffffu, s.l, o)};
        s = df_add(s, w);
      }
      if (lane == 0) {
        redf[2 * wid] = s.h;
        redf[2 * wid + 1] = s.l;
      }
    }
    __syncthreads();
    double tot = 0.0;
    if (tid == 0) {
      dfloat t{redf[0], redf[1]};
      for (int w = 1; w < W / 32; ++w) t = df_add(t, dfloat{redf[2 * w], redf[2 * w + 1]});
      tot = (double)t.h + (double)t.l;
    }
    __syncthreads();
    return tot;
  } else {
    double s = 0.0;
    if (tid < W) {
      for (int b0 = tid; b0 < n; b0 += UN * W) {
        double x[UN];
#pragma unroll
        for (int j = 0; j < UN; ++j) x[j] = b0 + j * W < n ? __ldcg(partials + b0 + j * W) : 0.0;
#pragma unroll
        for (int j = 0; j < UN; ++j)
          if (b0 + j * W < n) s += x[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) red[wid] = s;
    }
    __syncthreads();
    double tot = 0.0;
    if (tid == 0) {
      tot = red[0];
      for (int w = 1; w < W / 32; ++w) tot += red[w];
    }
    __syncthreads();
    return tot;
  }
}

static __device__ __forceinline__ int vol_readi(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Per-thread accumulator of a block reduction: double-float for float
// kernels (no FP64 instruction), double for the FP64 path.
template <>
struct Acc<float> {
  dfloat v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = df_add(v, x); }
  __device__ __forceinline__ double block_total(float* scr_f, double*) { return block_sum_df(v, scr_f); }
};
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double block_total(float*, double* scr_d) {
    double a[1] = {v};
    block_sum<1>(a, scr_d);
    return a[0];
  }
};

template <>
__device__ __forceinline__ void store_deferred_partial<float>(Acc<float>& acc, double* slot, float* redf, double*) {
  const dfloat t = block_sum_df2(acc.v, redf);
  if (flat_tid() == 0) *reinterpret_cast<float2*>(slot) = make_float2(t.h, t.l);
}
template <>
__device__ __forceinline__ void store_deferred_partial<double>(Acc<double>& acc, double* slot, float*, double* red) {
  const double t = acc.block_total(nullptr, red);
  if (flat_tid() == 0) *slot = t;
}

// A column / line pass runs for problem b in this mode: ITER and TRUE skip
// converged problems, RESTART runs only for the problems being restarted.
static __device__ __forceinline__ bool col_active(int mode, const int* pmode, const SolverScalars* sc) {
  if (mode == COL_RESTART) return pmode && *pmode == 2;
  if (mode == COL_ITER || mode == COL_TRUE) return !done_flag(sc);
  if (mode == COL_TRUENORM) return unchecked_stop(sc);  // the gate's true residuals: newly stopped problems
  return true;
}

}  // namespace fftmech
