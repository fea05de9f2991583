// Control kernels of the device-driven PCG (no counterpart in the paper's
// method; they replace the host's convergence polling so that a whole solve
// or staggered step can run as one CUDA graph): solver-scalar set-up, the
// zero right-hand-side case, loop decisions of batches, the restart gate
// after a recursive convergence, and device timestamps.
#include "fftmech_internal.cuh"
#include "fftmech.h"
#include "pcg_dev.cuh"

namespace fftmech {

static constexpr int kCtlThreads = 256;

// Fresh scalars for every problem of a solve.
__global__ void k_sc_init(SolverScalars* sc, int batch, double tol2, int max_iter, int reliable) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    SolverScalars s;
    memset(&s, 0, sizeof(s));
    s.tol2 = tol2;
    s.max_iter = max_iter;
    s.reliable = reliable;
    sc[b] = s;
  }
}

// After the first residual: a zero right-hand side (<f, M^-1 f> = 0) with a
// non-zero warm start has the solution u = 0 (0 iterations). With a
// Dirichlet mask that case is an argument error. n = D N iterate values per
// problem; grid.y = problem.
__global__ void k_zero_rhs(double* u, float* uh, float* ul, long long n, SolverScalars* sc, int has_mask) {
  const int b = blockIdx.y;
  SolverScalars* s = sc + b;
  const double rz0 = vol_read(&s->rz0), rz = vol_read(&s->rz);
  if (!(rz0 == 0.0 && rz > 0.0)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->done = 1;
    s->status = has_mask ? FFTMECH_ERR_INVALID_ARG : FFTMECH_OK;
  }
  if (has_mask) return;
  const size_t o = (size_t)b * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    u[o + i] = 0.0;
    if (uh) {
      uh[o + i] = 0.f;
      ul[o + i] = 0.f;
    }
  }
}

// Loop decisions of a batch after a direction (the direction kernel takes
// them itself for one problem): ordinary iterations continue while some
// problem is active and none replaces its residual next; a replacement
// iteration (which the others run as an ordinary one) comes first
// otherwise; the gate's true-residual passes run when some problem has
// stopped unchecked.
__global__ void __launch_bounds__(kCtlThreads) k_loopctl(const SolverScalars* sc, const int* mode, int batch,
                                                         LoopCtl ctl) {
  int active = 0, rep = 0, gate = 0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const int a = !done_flag(sc + b);
    active |= a;
    if (a && mode && vol_readi(mode + b) == 1) rep = 1;
    if (unchecked_stop(sc + b)) gate = 1;
  }
  active = __syncthreads_or(active);
  rep = __syncthreads_or(rep);
  gate = __syncthreads_or(gate);
  if (threadIdx.x == 0) loop_decide(ctl, active, rep, gate);
}

// End of an outer round. Problems that stopped in this round have their
// FP64 true residuals in rz_true now and are marked checked (later rounds
// skip their true-residual pass). While some problem is still active (a
// replacement iteration ended the round) the solve goes on.
// Once all have stopped: a
// problem whose recursive residual met tol while its true residual did not
// continues from the true residual with a fresh direction (mode 2), at most
// three times and within max_iter; LF_OUTER = LF_RESTART = some problem
// restarts. A solve whose rounds exceed max_rounds (a guard: every round
// ends an iteration or a restart) stops with its active problems marked
// not converged.
__global__ void __launch_bounds__(kCtlThreads) k_gate(SolverScalars* sc, int* mode, int batch, LoopCtl ctl,
                                                      int max_rounds) {
  __shared__ int rounds;
  if (threadIdx.x == 0) {
    rounds = ctl.flags ? ctl.flags[LF_ROUNDS] + 1 : 0;
    if (ctl.flags) ctl.flags[LF_ROUNDS] = rounds;
  }
  __syncthreads();
  int active = 0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    if (done_flag(sc + b)) sc[b].checked = 1;
    else active = 1;
  }
  active = __syncthreads_or(active);
  if (active && rounds > max_rounds) {
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
      if (!done_flag(sc + b)) {
        sc[b].status = FFTMECH_ERR_NOT_CONVERGED;
        sc[b].done = 1;
      }
      mode[b] = 0;
    }
    if (threadIdx.x == 0) {
      set_loop_flag(ctl, LF_OUTER, 0);
      set_loop_flag(ctl, LF_RESTART, 0);
    }
    return;
  }
  if (active) {
    if (threadIdx.x == 0) {
      set_loop_flag(ctl, LF_OUTER, 1);
      set_loop_flag(ctl, LF_RESTART, 0);
    }
    return;
  }
  int any = 0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    SolverScalars* s = sc + b;
    const bool gate = s->reliable && s->status == FFTMECH_OK && s->nrestart < 3 && s->iter < s->max_iter &&
                      s->rz_true > s->tol2 * s->rz0;
    mode[b] = gate ? 2 : 0;
    if (gate) {
      s->done = 0;
      s->checked = 0;
      s->nrestart += 1;
      any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    set_loop_flag(ctl, LF_OUTER, any);
    set_loop_flag(ctl, LF_RESTART, any);
  }
}

// Start of an outer round: the loop, replacement and gate conditions take
// the values the last decision stored in device memory.
__global__ void k_sync_flags(LoopCtl ctl) {
  if (threadIdx.x != 0 || !ctl.flags) return;
  set_loop_flag(ctl, LF_LOOP, vol_readi(ctl.flags + LF_LOOP));
  set_loop_flag(ctl, LF_REPLACE, vol_readi(ctl.flags + LF_REPLACE));
  set_loop_flag(ctl, LF_GATE, vol_readi(ctl.flags + LF_GATE));
}

// Restarted problems return to ordinary iterations.
__global__ void k_clear_modes(int* mode, int batch) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x)
    if (mode[b] == 2) mode[b] = 0;
}

// Sets flag k (and zeroes the round counter when k is LF_OUTER, the start of
// a solve).
__global__ void k_set_flag(LoopCtl ctl, int k, int value) {
  if (threadIdx.x != 0) return;
  set_loop_flag(ctl, k, value);
  if (k == LF_OUTER && ctl.flags) ctl.flags[LF_ROUNDS] = 0;
}

// Device clock (ns) at the point the stream reaches this launch.
__global__ void k_stamp(unsigned long long* slot) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  if (threadIdx.x == 0) *slot = t;
}

cudaError_t launch_sc_init(SolverScalars* sc, int batch, double tol2, int max_iter, int reliable, cudaStream_t st) {
  k_sc_init<<<(batch + kCtlThreads - 1) / kCtlThreads, kCtlThreads, 0, st>>>(sc, batch, tol2, max_iter, reliable);
  return cudaGetLastError();
}

cudaError_t launch_zero_rhs(double* u, float* uh, float* ul, long long n, SolverScalars* sc, int batch, int has_mask,
                            cudaStream_t st) {
  long long g = (n + kCtlThreads - 1) / kCtlThreads;
  if (g > 1024) g = 1024;
  k_zero_rhs<<<dim3((unsigned)(g < 1 ? 1 : g), batch), kCtlThreads, 0, st>>>(u, uh, ul, n, sc, has_mask);
  return cudaGetLastError();
}

cudaError_t launch_loopctl(const SolverScalars* sc, const int* mode, int batch, const LoopCtl& ctl,
                           cudaStream_t st) {
  k_loopctl<<<1, kCtlThreads, 0, st>>>(sc, mode, batch, ctl);
  return cudaGetLastError();
}

cudaError_t launch_gate(SolverScalars* sc, int* mode, int batch, const LoopCtl& ctl, int max_rounds,
                        cudaStream_t st) {
  k_gate<<<1, kCtlThreads, 0, st>>>(sc, mode, batch, ctl, max_rounds);
  return cudaGetLastError();
}

cudaError_t launch_sync_flags(const LoopCtl& ctl, cudaStream_t st) {
  k_sync_flags<<<1, 32, 0, st>>>(ctl);
  return cudaGetLastError();
}

cudaError_t launch_clear_modes(int* mode, int batch, cudaStream_t st) {
  k_clear_modes<<<(batch + kCtlThreads - 1) / kCtlThreads, kCtlThreads, 0, st>>>(mode, batch);
  return cudaGetLastError();
}

cudaError_t launch_set_flag(const LoopCtl& ctl, int k, int value, cudaStream_t st) {
  k_set_flag<<<1, 32, 0, st>>>(ctl, k, value);
  return cudaGetLastError();
}

cudaError_t launch_stamp(unsigned long long* slot, cudaStream_t st) {
  k_stamp<<<1, 32, 0, st>>>(slot);
  return cudaGetLastError();
}

}  // namespace fftmech
