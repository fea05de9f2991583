// C ABI of libfftmech: contexts, FFT plans, workspace, the PCG loop and the
// entry points declared in include/fftmech.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "fftmech.h"
#include "fftmech_internal.cuh"
#include "host_plan.cuh"

using namespace fftmech;

namespace fftmech {
thread_local int tl_dependent_launch = 0;
}

namespace {

constexpr int kMaxBlocks = 8192;     // upper bound on reduction partials per launch
constexpr int kPartialSlots = 16;    // doubles per block in `partials`

// ---------------------------------------------------------------- plans
// Device twiddles for a context (FP64 values from the host, also rounded to
// float).
// Device buffers of a plan: twiddles (tw_smem_twiddles bytes) followed by
// the pass multipliers, tw_smem_bytes in all, for float and double.
template <typename T>
cudaError_t upload_plan(const HostPlan& p, const cx<double>* hd, cx<T>** dst) {
  const size_t bytes = tw_smem_bytes<T>(p.n), twb = tw_smem_twiddles<T>(p.n);
  std::vector<unsigned char> buf(bytes, 0);
  cx<T>* tw = reinterpret_cast<cx<T>*>(buf.data());
  for (int i = 0; i < p.n - 1; ++i) {
    tw[i].re = (T)hd[i].re;
    tw[i].im = (T)hd[i].im;
  }
  plan_multipliers(p.n, p.npass, p.radix, reinterpret_cast<unsigned int*>(buf.data() + twb));
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, buf.data(), bytes, cudaMemcpyHostToDevice);
}

cudaError_t make_plan(int n, HostPlan& p) {
  factor_plan(n, p);
  std::vector<cx<double>> hd(std::max(n, 1));
  fill_twiddles(p, hd.data());
  cudaError_t e = upload_plan<float>(p, hd.data(), &p.tw_f);
  if (e != cudaSuccess) return e;
  return upload_plan<double>(p, hd.data(), &p.tw_d);
}

void free_plan(HostPlan& p) {
  if (p.tw_f) cudaFree(p.tw_f);
  if (p.tw_d) cudaFree(p.tw_d);
  p.tw_f = nullptr;
  p.tw_d = nullptr;
}

}  // namespace

// ---------------------------------------------------------------- context
struct Staging {
  void* dev = nullptr;
  size_t bytes = 0;
};

enum StageSlot {
  ST_PHASE, ST_EIG, ST_DAMAGE, ST_U, ST_STRAIN, ST_STRESS, ST_C, ST_H, ST_MASK, ST_CPPT,
  ST_EIGFIELD, ST_COUNT
};

struct fftmech_ctx {
  int dim = 2;
  int nx = 1, ny = 1, nz = 1;
  long long N = 0;  // voxels of one problem
  int B = 1;        // problems in the (uniform) batch
  double h = 1, h_diff = 1;
  fftmech_materials mat{};
  fftmech_precision prec = FFTMECH_FP64;
  fftmech_solver_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int nsm = 0;
  size_t optin = 0;
  HostPlan px, py, pz;
  Shape2 shape{};
  Shape3 shape3{};
  LineShape lshape{};
  StenShape sshape{};
  // workspace (B problems back to back)
  void* r = nullptr;
  void* p[2] = {nullptr, nullptr};
  void* S = nullptr;
  void* q = nullptr;     // K p of the split iteration
  void* g = nullptr;
  float* uh = nullptr;   // MIXED iterate, high part
  float* ul = nullptr;   // MIXED iterate, low part
  double* phi = nullptr;
  double* Hd = nullptr;
  double* cn = nullptr;
  void* lamx = nullptr;
  void* lamy = nullptr;
  void* lamz = nullptr;     // 3D: lambda_z(kz)
  void* lamc3 = nullptr;    // 3D: lambda_x per spectral column, D = 3 / D = 1 rows
  void* lamc1 = nullptr;
  void* wcol3 = nullptr;    // 3D: Parseval weight per spectral column
  void* wcol1 = nullptr;
  double* partials = nullptr;
  double* partials_col = nullptr;  // 2D column pass (deferred reductions)
  double* results = nullptr;   // 16 per problem
  double* m0b = nullptr;       // per-problem preconditioner constants
  double* m1b = nullptr;
  int* mode = nullptr;         // per-problem reliable-update / restart flags
  SolverScalars* sc = nullptr;
  SolverScalars* h_sc = nullptr;   // pinned
  double* h_results = nullptr;     // pinned
  int* h_mode = nullptr;           // host copy of the modes, edited freely
  // pinned ring the mode pushes copy from: an asynchronous copy reads its
  // pinned source when it runs, so a slot is reused only after its copy ran
  static constexpr int kModeSlots = 4;
  int* h_mode_ring = nullptr;
  cudaEvent_t mode_ev[kModeSlots] = {nullptr, nullptr, nullptr, nullptr};
  int mode_slot = 0;
  Staging stage[ST_COUNT];
  // instrumentation
  bool prof = false;
  long long launches[FFTMECH_K_COUNT] = {0};
  double prof_ms[FFTMECH_K_COUNT] = {0};
  struct Pending { int k; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  cudaEvent_t solve_ev[2] = {nullptr, nullptr};
  char err[512] = {0};
};

namespace {

constexpr int kResultsPerProblem = 16;

fftmech_status set_err(fftmech_ctx* ctx, fftmech_status s, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

#define CK(expr)                                                                      \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess)                                                            \
      return set_err(ctx, FFTMECH_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

size_t esize(const fftmech_ctx* ctx) { return ctx->prec == FFTMECH_FP64 ? 8 : 4; }
int nvoigt(const fftmech_ctx* ctx) { return ctx->dim == 2 ? 3 : 6; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller buffer: the pointer itself if it is device memory,
// else a staging buffer (copied in when `in`). Output copy-back is done by
// `stage_out`.
fftmech_status stage_in(fftmech_ctx* ctx, StageSlot slot, const void* ptr, size_t bytes, bool in,
                        void** dev) {
  if (!ptr) { *dev = nullptr; return FFTMECH_OK; }
  if (is_device_ptr(ptr)) { *dev = const_cast<void*>(ptr); return FFTMECH_OK; }
  Staging& s = ctx->stage[slot];
  if (s.bytes < bytes) {
    if (s.dev) CK(cudaFree(s.dev));
    s.dev = nullptr;
    s.bytes = 0;
    if (cudaMalloc(&s.dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, FFTMECH_ERR_OOM, "staging buffer of %zu bytes", bytes);
    }
    s.bytes = bytes;
  }
  if (in) CK(cudaMemcpyAsync(s.dev, ptr, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *dev = s.dev;
  return FFTMECH_OK;
}

fftmech_status stage_out(fftmech_ctx* ctx, void* host, const void* dev, size_t bytes) {
  if (!host || host == dev) return FFTMECH_OK;
  CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return FFTMECH_OK;
}

// ---------------------------------------------------------------- instrumentation
cudaEvent_t take_event(fftmech_ctx* ctx) {
  if (!ctx->ev_free.empty()) {
    cudaEvent_t e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Counts one launch of class k and, when profiling, brackets it with events.
struct ProfScope {
  fftmech_ctx* ctx;
  int k;
  cudaEvent_t a = nullptr;
  ProfScope(fftmech_ctx* c, int kc) : ctx(c), k(kc) {
    ctx->launches[k] += 1;
    if (ctx->prof) {
      a = take_event(ctx);
      if (a) cudaEventRecord(a, ctx->stream);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    if (!b) { ctx->ev_free.push_back(a); return; }
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({k, a, b});
  }
};

// After a stream synchronisation: fold the completed event pairs into the
// per-class totals and recycle the events.
void prof_flush(fftmech_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->prof_ms[p.k] += ms;
    else cudaGetLastError();
    ctx->ev_free.push_back(p.a);
    ctx->ev_free.push_back(p.b);
  }
  ctx->pending.clear();
}

#define FFTMECH_LAUNCH(KC, CALL) \
  do {                           \
    ProfScope _ps(ctx, KC);      \
    CK(CALL);                    \
  } while (0)

void lame(double E, double nu, double& lam, double& mu) {
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  mu = E / (2.0 * (1.0 + nu));
}

fftmech_status sync_scalars(fftmech_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(SolverScalars) * ctx->B, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FFTMECH_OK;
}

fftmech_status push_modes(fftmech_ctx* ctx) {
  const int k = ctx->mode_slot;
  ctx->mode_slot = (k + 1) % fftmech_ctx::kModeSlots;
  CK(cudaEventSynchronize(ctx->mode_ev[k]));  // the slot's previous copy has run
  int* slot = ctx->h_mode_ring + (size_t)k * ctx->B;
  std::memcpy(slot, ctx->h_mode, sizeof(int) * ctx->B);
  CK(cudaMemcpyAsync(ctx->mode, slot, sizeof(int) * ctx->B, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaEventRecord(ctx->mode_ev[k], ctx->stream));
  return FFTMECH_OK;
}

// ---------------------------------------------------------------- PCG loop
struct Solve {
  int iters = 0;
  int status = FFTMECH_OK;
  double rel = 0, true_rel = 0;
};

// Preconditioned CG on the potential for every problem of the batch (see
// the kernels for the per-iteration launches). The host polls the device
// scalars every check_every iterations; a problem that has converged (or
// failed) stops moving while the others continue. MIXED: the iterate is a
// float pair, with reliable updates and a final FP64 true-residual gate.
template <typename T, int D>
fftmech_status run_pcg(fftmech_ctx* ctx, const Op<T>& op_in, double* u, const Spec<T>& sp_in,
                       std::vector<Solve>& out) {
  const DepLaunchScope dep(ctx->opts.launch_mode == 0);
  cudaStream_t st = ctx->stream;
  const int B = ctx->B;
  const Shape2& sh = ctx->shape;
  FftPlanDev<T> px = dev_plan<T>(ctx->px), py = dev_plan<T>(ctx->py);
  Spec<T> sp = sp_in;
  sp.lamx = (const T*)ctx->lamx;
  sp.lamy = (const T*)ctx->lamy;
  sp.invN = 1.0 / (double)ctx->N;
  sp.m0_t = (T)sp.m0;
  sp.m1_t = (T)sp.m1;
  sp.invN_t = (T)sp.invN;
  Op<T> op = op_in;  // with the constants rounded to T
  op.ih_t = (T)(1.0 / op.h);
  for (int k = 0; k < 2; ++k) {
    op.lam_t[k] = (T)op.lam[k];
    op.mu_t[k] = (T)op.mu[k];
    op.kap_t[k] = (T)op.kap[k];
  }
  op.c0c_t = (T)op.c0c;
  for (int b = 0; b < B; ++b) {
    SolverScalars h{};
    h.tol2 = ctx->opts.tol * ctx->opts.tol;
    h.max_iter = ctx->opts.max_iter;
    ctx->h_sc[b] = h;
    ctx->h_mode[b] = 0;
  }
  CK(cudaMemcpyAsync(ctx->sc, ctx->h_sc, sizeof(SolverScalars) * B, cudaMemcpyHostToDevice, st));
  if (push_modes(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
  T* pbuf[2] = {(T*)ctx->p[0], (T*)ctx->p[1]};
  Vec2<T> v{};
  v.u = u;
  v.uh = ctx->uh;
  v.ul = ctx->ul;
  v.r = (T*)ctx->r;
  v.p_in = pbuf[0];
  v.p_out = pbuf[1];
  v.S = (cx<T>*)ctx->S;
  v.q = (T*)ctx->q;
  v.partials = ctx->partials;
  v.sc = ctx->sc;
  v.mode = ctx->mode;
  // Deferred reductions where the grid is latency-bound (up to 2^21 voxels
  // per launch): the stencil's <p, K p> summed by the update kernel (2D and
  // 3D), the column pass's <r, M^-1 r> by the next direction kernel (2D).
  // Larger grids keep the last-block reductions: there every consumer block
  // re-reading all partials costs more than the ticket saves.
  const bool small = (long long)ctx->N * B <= (1LL << 21);
  const bool defer = small && ctx->dim == 2;
  const int ncol_blocks = defer ? (ctx->nx + ctx->shape.cols - 1) / ctx->shape.cols : 0;
  v.pcol = ctx->partials_col;
  v.nsten = !small ? 0
            : ctx->dim == 2 ? sten2_blocks(ctx->nx, ctx->ny, ctx->sshape)
                            : sten3_blocks(ctx->nx, ctx->ny, ctx->nz, ctx->sshape);
  const long long nU = (long long)D * ctx->N * B;
  const bool mixed = sizeof(T) == 4;
  if (mixed) FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_df_split(nU, u, ctx->uh, ctx->ul, st));
  const int nx = ctx->nx, ny = ctx->ny;
  const int fx = ctx->px.fam, fy = ctx->py.fam, fz = ctx->pz.fam;
  const bool three = ctx->dim == 3;
  const Shape3& sh3 = ctx->shape3;
  FftPlanDev<T> pz = dev_plan<T>(ctx->pz);
  if (three) {
    sp.lamc = (const T*)(D == 1 ? ctx->lamc1 : ctx->lamc3);
    sp.wcol = (const T*)(D == 1 ? ctx->wcol1 : ctx->wcol3);
    sp.lamj = (const T*)ctx->lamy;
    sp.laml = (const T*)ctx->lamz;
  }
  auto residual = [&](int zero_u, int filter) -> cudaError_t {
    if constexpr (D == 3) return launch3_residual_f<T, 3>(fx, op, v, px, sh3, zero_u, filter, st);
    else if constexpr (D == 2) return launch_residual_f<T, 2>(fx, op, v, px, sh, zero_u, filter, st);
    else
      return three ? launch3_residual_f<T, 1>(fx, op, v, px, sh3, zero_u, filter, st)
                   : launch_residual_f<T, 1>(fx, op, v, px, sh, zero_u, filter, st);
  };
  // split iteration: x-line IFFT + direction, stencil q = K p + alpha,
  // x-line update + FFT
  const LineShape& lsh = ctx->lshape;
  const StenShape& ssh = ctx->sshape;
  auto direction = [&](const Vec2<T>& va) -> cudaError_t {
    if constexpr (D == 3) return launch_xdir_f<T, 3, 3>(fx, op, va, px, lsh, st);
    else if constexpr (D == 2) return launch_xdir_f<T, 2, 2>(fx, op, va, px, lsh, st);
    else
      return three ? launch_xdir_f<T, 1, 3>(fx, op, va, px, lsh, st) : launch_xdir_f<T, 1, 2>(fx, op, va, px, lsh, st);
  };
  auto stencil = [&](const Vec2<T>& vs) -> cudaError_t {
    if constexpr (D == 3) return launch_sten3<T, 3>(op, vs, ssh, st);
    else if constexpr (D == 2) return launch_sten2<T, 2>(op, vs, ssh, st);
    else return three ? launch_sten3<T, 1>(op, vs, ssh, st) : launch_sten2<T, 1>(op, vs, ssh, st);
  };
  auto update = [&](const Vec2<T>& vb) -> cudaError_t {
    if constexpr (D == 3) return launch_xupd_f<T, 3, 3>(fx, op, vb, px, lsh, st);
    else if constexpr (D == 2) return launch_xupd_f<T, 2, 2>(fx, op, vb, px, lsh, st);
    else
      return three ? launch_xupd_f<T, 1, 3>(fx, op, vb, px, lsh, st) : launch_xupd_f<T, 1, 2>(fx, op, vb, px, lsh, st);
  };
  // 2D: one column pass; 3D: y-FFT, z pass (multiplier, <r, M^-1 r>), y-IFFT
  auto colpass = [&](int mode) -> cudaError_t {
    if (!three)
      return launch_colpass_f<T>(fy, nx, ny, v.S, py, sp, sh, mode, 0, ctx->partials_col, ctx->sc, ctx->mode, st);
    cudaError_t e = launch3_lines_f<T>(fy, v.S, sh3, D, 1, 0, py, sp, mode, nullptr, ctx->sc, ctx->mode, st);
    if (e != cudaSuccess) return e;
    e = launch3_lines_f<T>(fz, v.S, sh3, D, 2, 1, pz, sp, mode, ctx->partials, ctx->sc, ctx->mode, st);
    if (e != cudaSuccess || mode == COL_NORM || mode == COL_TRUENORM) return e;
    return launch3_lines_f<T>(fy, v.S, sh3, D, 1, 2, py, sp, mode, nullptr, ctx->sc, ctx->mode, st);
  };
  FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, residual(1, 0));
  FFTMECH_LAUNCH(FFTMECH_K_COLUMN, colpass(COL_NORM));
  FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, residual(0, 0));
  FFTMECH_LAUNCH(FFTMECH_K_COLUMN, colpass(COL_INIT));
  if (sync_scalars(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
  // a zero right-hand side has the zero solution (outside Dirichlet voxels)
  for (int b = 0; b < B; ++b) {
    const SolverScalars& q = ctx->h_sc[b];
    if (q.rz0 == 0.0 && q.rz > 0.0) {
      if (op.mask) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "zero right-hand side with a Dirichlet mask");
      CK(cudaMemsetAsync(u + (size_t)b * D * ctx->N, 0, sizeof(double) * D * ctx->N, st));
      if (mixed) {
        CK(cudaMemsetAsync(ctx->uh + (size_t)b * D * ctx->N, 0, sizeof(float) * D * ctx->N, st));
        CK(cudaMemsetAsync(ctx->ul + (size_t)b * D * ctx->N, 0, sizeof(float) * D * ctx->N, st));
      }
      SolverScalars z = q;
      z.done = 1;
      z.status = FFTMECH_OK;
      z.rz = 0.0;
      CK(cudaMemcpyAsync(ctx->sc + b, &z, sizeof(SolverScalars), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
      ctx->h_sc[b] = z;
    }
  }
  const int check = std::max(1, ctx->opts.check_every);
  const bool reliable = mixed && ctx->opts.replace_residual != 0;
  std::vector<double> rz_rep(B);
  for (int b = 0; b < B; ++b) rz_rep[b] = ctx->h_sc[b].rz;
  auto all_done = [&]() {
    for (int b = 0; b < B; ++b)
      if (!ctx->h_sc[b].done) return false;
    return true;
  };
  bool pending = false;  // some problem has mode 1 queued for the next iteration
  bool col_deferred = false;  // the last column pass left its reduction to the next direction kernel
  int pi = 0;
  int it = 0;
  for (int restart = 0;; ++restart) {
    while (!all_done() && it < ctx->opts.max_iter) {
      Vec2<T> va = v;
      va.p_in = pbuf[pi];
      va.p_out = pbuf[1 - pi];
      va.ncol = col_deferred ? ncol_blocks : 0;
      FFTMECH_LAUNCH(FFTMECH_K_DIRECTION, direction(va));
      Vec2<T> vb = v;
      vb.p_in = pbuf[1 - pi];
      vb.defer_rz = col_deferred ? 1 : 0;
      FFTMECH_LAUNCH(FFTMECH_K_STENCIL, stencil(vb));
      FFTMECH_LAUNCH(FFTMECH_K_UPDATE, update(vb));
      const bool replace = pending;
      // reliable update: u += alpha p only (update kernel), then the FP64 true residual
      if (replace) FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, residual(0, 1));
      // a replacement iteration finalises at once (the host reads rz_true next)
      col_deferred = defer && !replace;
      FFTMECH_LAUNCH(FFTMECH_K_COLUMN, colpass(col_deferred ? (COL_ITER | COL_DEFER) : COL_ITER));
      pi = 1 - pi;
      ++it;
      if (replace) {
        for (int b = 0; b < B; ++b) ctx->h_mode[b] = 0;
        if (push_modes(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
        pending = false;
      }
      if (it % check == 0 || it >= ctx->opts.max_iter || replace) {
        if (sync_scalars(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
        bool any = false;
        for (int b = 0; b < B; ++b) {
          const SolverScalars& q = ctx->h_sc[b];
          if (replace) rz_rep[b] = q.rz_true > 0 ? q.rz_true : rz_rep[b];
          if (reliable && !replace && !q.done && q.rz < 1e-2 * rz_rep[b]) {
            ctx->h_mode[b] = 1;
            any = true;
          }
        }
        if (any) {
          if (push_modes(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
          pending = true;
        }
      }
    }
    // the iteration limit stopped the loop right after a deferred column pass
    if (col_deferred) {
      FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_col_finalize(ctx->partials_col, ncol_blocks, ctx->sc, B,
                                                          1.0 / (double)ctx->N, mixed ? 1 : 0, st));
      col_deferred = false;
    }
    // FP64 true residual of every iterate
    FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, residual(0, 0));
    FFTMECH_LAUNCH(FFTMECH_K_COLUMN, colpass(COL_TRUENORM));
    if (sync_scalars(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
    // problems whose float recursion met tol while the FP64 true residual did
    // not: continue from the true residual with a fresh direction (at most
    // three restarts)
    bool any = false;
    for (int b = 0; b < B; ++b) {
      const SolverScalars& q = ctx->h_sc[b];
      const bool gate = reliable && q.status == FFTMECH_OK && restart < 3 && q.iter < ctx->opts.max_iter &&
                        q.rz_true > q.tol2 * q.rz0;
      ctx->h_mode[b] = gate ? 2 : 0;
      if (gate) {
        const int zero = 0;
        CK(cudaMemcpyAsync(&ctx->sc[b].done, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
        any = true;
      }
    }
    if (!any) break;
    if (push_modes(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
    FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, residual(0, 1));
    FFTMECH_LAUNCH(FFTMECH_K_COLUMN, colpass(COL_RESTART));
    for (int b = 0; b < B; ++b) ctx->h_mode[b] = 0;
    if (push_modes(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
    if (sync_scalars(ctx) != FFTMECH_OK) return FFTMECH_ERR_CUDA;
    for (int b = 0; b < B; ++b) rz_rep[b] = ctx->h_sc[b].rz;
    pending = false;
  }
  if (mixed) FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_df_merge(nU, ctx->uh, ctx->ul, u, st));
  out.assign(B, Solve());
  for (int b = 0; b < B; ++b) {
    const SolverScalars& f = ctx->h_sc[b];
    out[b].iters = f.iter;
    out[b].status = f.done ? f.status : FFTMECH_ERR_NOT_CONVERGED;
    out[b].rel = f.rz0 > 0 ? std::sqrt(std::max(f.rz, 0.0) / f.rz0) : 0.0;
    out[b].true_rel = f.rz0 > 0 ? std::sqrt(std::max(f.rz_true, 0.0) / f.rz0) : 0.0;
  }
  return FFTMECH_OK;
}

template <typename T>
void base_op(const fftmech_ctx* ctx, Op<T>& op, const uint8_t* phase) {
  std::memset(&op, 0, sizeof(op));
  op.nx = ctx->nx;
  op.ny = ctx->ny;
  op.nz = ctx->nz;
  op.h = ctx->h;
  op.phase = phase;
  lame(ctx->mat.E_pore, ctx->mat.nu_pore, op.lam[0], op.mu[0]);
  lame(ctx->mat.E_solid, ctx->mat.nu_solid, op.lam[1], op.mu[1]);
  op.src_scale = 1.0;
}

fftmech_status read_results(fftmech_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_results, ctx->results, sizeof(double) * kResultsPerProblem * ctx->B,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FFTMECH_OK;
}

// Device time of one solve: events at its start and end on the context stream.
fftmech_status solve_timer_start(fftmech_ctx* ctx) {
  CK(cudaEventRecord(ctx->solve_ev[0], ctx->stream));
  return FFTMECH_OK;
}
fftmech_status solve_timer_stop(fftmech_ctx* ctx) {
  CK(cudaEventRecord(ctx->solve_ev[1], ctx->stream));
  return FFTMECH_OK;
}
double solve_timer_ms(fftmech_ctx* ctx) {
  float ms = 0.f;
  if (cudaEventSynchronize(ctx->solve_ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&ms, ctx->solve_ev[0], ctx->solve_ev[1]) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return (double)ms;
}

// Per-problem info records sit `stride` apart (1 for single solves, 3 in a
// staggered step).
fftmech_solve_info& info_at(fftmech_solve_info* info, int b, int stride) { return info[(size_t)b * stride]; }

fftmech_status worst_status(const std::vector<Solve>& s) {
  fftmech_status w = FFTMECH_OK;
  for (const Solve& x : s)
    if (x.status != FFTMECH_OK && w == FFTMECH_OK) w = (fftmech_status)x.status;
  return w;
}

void copy_solves(const std::vector<Solve>& s, fftmech_solve_info* info, int stride, double ms) {
  for (size_t b = 0; b < s.size(); ++b) {
    fftmech_solve_info& i = info_at(info, (int)b, stride);
    i.status = s[b].status;
    i.iters = s[b].iters;
    i.rel_res = s[b].rel;
    i.true_rel_res = s[b].true_rel;
    i.device_ms = ms;
  }
}

// ---------------------------------------------------------------- solves
template <typename T>
fftmech_status equilibrium_impl(fftmech_ctx* ctx, const uint8_t* phase, const T* eig,
                                const double* damage, const double* eps_mac, double* u, T* strain,
                                T* stress, fftmech_solve_info* info, int stride) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc = solve_timer_start(ctx);
  if (rc != FFTMECH_OK) return rc;
  const int B = ctx->B;
  const long long NB = ctx->N * B;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  op.eig = eig;
  for (int k = 0; k < nvoigt(ctx); ++k) op.E[k] = eps_mac[k];
  if (damage) {
    FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_degradation<T>(NB, damage, ctx->mat.kappa, (T*)ctx->g, st));
    op.g = (const T*)ctx->g;
  }
  Spec<T> sp{};
  sp.m0 = 0.0;
  sp.m1 = 1.0 / (ctx->h * ctx->h);
  std::vector<Solve> s;
  const bool three = ctx->dim == 3;
  rc = three ? run_pcg<T, 3>(ctx, op, u, sp, s) : run_pcg<T, 2>(ctx, op, u, sp, s);
  if (rc != FFTMECH_OK) return rc;
  if (three)
    FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch3_el_output<T>(op, B, u, strain, stress, ctx->partials, ctx->results, ctx->sc, st));
  else
    FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_el_output<T>(op, B, u, strain, stress, ctx->partials, ctx->results, ctx->sc, st));
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  if ((rc = read_results(ctx)) != FFTMECH_OK) return rc;
  const double ms = solve_timer_ms(ctx);
  copy_solves(s, info, stride, ms);
  const double N = (double)ctx->N;
  const int nv = nvoigt(ctx);
  const double vox = three ? ctx->h * ctx->h * ctx->h : ctx->h * ctx->h;
  for (int b = 0; b < B; ++b) {
    const double* R = ctx->h_results + b * (2 * nv + 1);
    fftmech_solve_info& i = info_at(info, b, stride);
    for (int k = 0; k < nv; ++k) {
      i.mean_stress[k] = R[k] / N;
      i.mean_strain[k] = R[nv + k] / N;
    }
    i.elastic_energy = R[2 * nv] * vox;
  }
  return worst_status(s);
}

template <typename T>
fftmech_status diffusion_impl(fftmech_ctx* ctx, const uint8_t* phase, int mode,
                              const double* grad_c_mac, double c_macro, double dt,
                              const uint8_t* mask, double cD, double* c,
                              fftmech_solve_info* info, int stride) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc = solve_timer_start(ctx);
  if (rc != FFTMECH_OK) return rc;
  const int B = ctx->B;
  const long long NB = ctx->N * B;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  op.h = ctx->h_diff;
  op.kap[0] = ctx->mat.D_pore;
  op.kap[1] = ctx->mat.D_solid;
  const double ih2 = 1.0 / (ctx->h_diff * ctx->h_diff);
  std::vector<Solve> s;
  Spec<T> sp{};
  if (mode == FFTMECH_DIFF_HOMOGENISE) {
    const bool three = ctx->dim == 3;
    op.G[0] = grad_c_mac[0];
    op.G[1] = grad_c_mac[1];
    op.G[2] = three ? grad_c_mac[2] : 0.0;
    sp.m0 = 0.0;
    sp.m1 = ih2;
    rc = run_pcg<T, 1>(ctx, op, ctx->phi, sp, s);
    if (rc != FFTMECH_OK) return rc;
    if (three) {
      FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch3_diff_stats<T>(op, B, ctx->phi, ctx->h_diff, c_macro, ctx->partials,
                                                            ctx->results, ctx->sc, st));
      FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch3_diff_write_c(ctx->nx, ctx->ny, ctx->nz, B, phase, ctx->phi,
                                                           ctx->h_diff, op.G, ctx->results, c, st));
    } else {
      FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_diff_stats<T>(op, B, ctx->phi, ctx->h_diff, c_macro, ctx->partials,
                                                           ctx->results, ctx->sc, st));
      FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_diff_write_c(ctx->nx, ctx->ny, B, phase, ctx->phi, ctx->h_diff,
                                                          op.G[0], op.G[1], ctx->results, c, st));
    }
    if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
    if ((rc = read_results(ctx)) != FFTMECH_OK) return rc;
    copy_solves(s, info, stride, solve_timer_ms(ctx));
    const int nr = three ? 6 : 5, nd = three ? 3 : 2;
    for (int b = 0; b < B; ++b) {
      const double* R = ctx->h_results + b * nr;
      fftmech_solve_info& i = info_at(info, b, stride);
      for (int k = 0; k < nd; ++k) i.mean_flux[k] = R[2 + k];
      i.porosity = R[2 + nd];
      i.mean_c = c_macro;
    }
    return worst_status(s);
  }
  // TRANSIENT (backward Euler, not in the paper)
  if (!(dt > 0)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt must be > 0 for TRANSIENT");
  // per-problem porosity -> mean diffusivity of the preconditioner (on device)
  FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_pf_stats(ctx->N, B, phase, nullptr, ctx->partials, ctx->results, ctx->sc,
                                                  ctx->mat.D_pore, ctx->mat.D_solid, ih2, ctx->m1b, st));
  if (mask) FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_set_masked(NB, mask, cD, c, st));
  CK(cudaMemcpyAsync(ctx->cn, c, sizeof(double) * NB, cudaMemcpyDeviceToDevice, st));
  op.c0c = 1.0 / dt;
  op.srcd = ctx->cn;
  op.src_scale = 1.0 / dt;
  op.mask = mask;
  sp.m0 = 1.0 / dt;
  sp.m1b = ctx->m1b;
  rc = run_pcg<T, 1>(ctx, op, c, sp, s);
  if (rc != FFTMECH_OK) return rc;
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  if ((rc = read_results(ctx)) != FFTMECH_OK) return rc;
  copy_solves(s, info, stride, solve_timer_ms(ctx));
  for (int b = 0; b < B; ++b)
    info_at(info, b, stride).porosity = 1.0 - ctx->h_results[b * 3 + 2] / (double)ctx->N;
  return worst_status(s);
}

template <typename T>
fftmech_status phasefield_impl(fftmech_ctx* ctx, const T* strain, const T* eig,
                               const uint8_t* phase, T* H, double* d, fftmech_solve_info* info,
                               int stride) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc = solve_timer_start(ctx);
  if (rc != FFTMECH_OK) return rc;
  const int B = ctx->B;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  const double a = ctx->mat.Gc / (2.0 * ctx->mat.l0);
  const double b = ctx->mat.Gc * ctx->mat.l0 / 2.0;
  // history update; m0b[p] = a + mean(H) of each problem (on device)
  if (ctx->dim == 3)
    FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch3_history<T>(ctx->N, B, phase, op.lam[0], op.lam[1], op.mu[0], op.mu[1],
                                                       strain, eig, H, ctx->Hd, a, ctx->m0b, ctx->partials, ctx->sc,
                                                       st));
  else
    FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_history<T>(ctx->N, B, phase, op.lam[0], op.lam[1], op.mu[0], op.mu[1],
                                                      strain, eig, H, ctx->Hd, a, ctx->m0b, ctx->partials, ctx->sc,
                                                      st));
  op.kap[0] = op.kap[1] = b;
  op.c0c = a;
  op.c0f = H;
  op.srcd = ctx->Hd;
  op.src_scale = 1.0;
  Spec<T> sp{};
  sp.m0b = ctx->m0b;
  sp.m1 = b / (ctx->h * ctx->h);
  std::vector<Solve> s;
  rc = run_pcg<T, 1>(ctx, op, d, sp, s);
  if (rc != FFTMECH_OK) return rc;
  FFTMECH_LAUNCH(FFTMECH_K_OTHER, launch_pf_stats(ctx->N, B, phase, d, ctx->partials, ctx->results, ctx->sc,
                                                  0.0, 0.0, 0.0, nullptr, st));
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  if ((rc = read_results(ctx)) != FFTMECH_OK) return rc;
  copy_solves(s, info, stride, solve_timer_ms(ctx));
  for (int p = 0; p < B; ++p) {
    const double* R = ctx->h_results + p * 3;
    fftmech_solve_info& i = info_at(info, p, stride);
    i.total_damage = R[0];
    i.frac_damaged = R[2] > 0 ? R[1] / R[2] : 0.0;
  }
  return worst_status(s);
}

fftmech_status check_ctx(fftmech_ctx* ctx) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return set_err(ctx, FFTMECH_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return FFTMECH_OK;
}

// |D_alpha|^2 h^2 = 2 - 2 cos(2 pi k / n) per direction (Sec. 2.6, forward
// difference); 3D also the per-spectral-column tables of the line passes.
template <typename T>
fftmech_status fill_lam(fftmech_ctx* ctx) {
  auto sym = [](int k, int n) { return (T)(2.0 - 2.0 * std::cos(2.0 * M_PI * k / n)); };
  std::vector<T> lx(ctx->nx), ly(ctx->ny);
  for (int k = 0; k < ctx->nx; ++k) lx[k] = sym(k, ctx->nx);
  for (int k = 0; k < ctx->ny; ++k) ly[k] = sym(k, ctx->ny);
  CK(cudaMemcpy(ctx->lamx, lx.data(), sizeof(T) * ctx->nx, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->lamy, ly.data(), sizeof(T) * ctx->ny, cudaMemcpyHostToDevice));
  if (ctx->dim == 3) {
    const int nx = ctx->nx, nxh = nx / 2 + 1;
    std::vector<T> lz(ctx->nz), c3, c1, w3, w1;
    for (int k = 0; k < ctx->nz; ++k) lz[k] = sym(k, ctx->nz);
    // half-spectrum column kx counts for kx and nx - kx unless they coincide
    auto half_w = [&](int k) { return (T)((k == 0 || 2 * k == nx) ? 1.0 : 2.0); };
    for (int k = 0; k < nx; ++k) { c3.push_back(lx[k]); w3.push_back((T)1); }
    for (int k = 0; k < nxh; ++k) {
      c3.push_back(lx[k]); w3.push_back(half_w(k));
      c1.push_back(lx[k]); w1.push_back(half_w(k));
    }
    CK(cudaMemcpy(ctx->lamz, lz.data(), sizeof(T) * ctx->nz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->lamc3, c3.data(), sizeof(T) * c3.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->wcol3, w3.data(), sizeof(T) * w3.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->lamc1, c1.data(), sizeof(T) * c1.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->wcol1, w1.data(), sizeof(T) * w1.size(), cudaMemcpyHostToDevice));
  }
  return FFTMECH_OK;
}

bool is_hard_error(fftmech_status s) {
  return s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

const char* fftmech_status_string(int s) {
  switch (s) {
    case FFTMECH_OK: return "ok";
    case FFTMECH_ERR_INVALID_ARG: return "invalid argument";
    case FFTMECH_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case FFTMECH_ERR_NOT_CONVERGED: return "not converged";
    case FFTMECH_ERR_NONFINITE: return "non-finite residual";
    case FFTMECH_ERR_TIMEOUT: return "device wait timed out";
    case FFTMECH_ERR_CUDA: return "CUDA error";
    case FFTMECH_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

const char* fftmech_last_error(const fftmech_ctx* ctx) { return ctx ? ctx->err : ""; }

fftmech_status fftmech_create_batched(fftmech_ctx** out, const fftmech_grid* grid, int batch,
                                      const fftmech_materials* mat, fftmech_precision precision,
                                      const fftmech_solver_opts* opts, void* stream) {
  if (!out || !grid || !mat || !opts) return FFTMECH_ERR_INVALID_ARG;
  *out = nullptr;
  if (batch < 1) return FFTMECH_ERR_INVALID_ARG;
  if (precision != FFTMECH_FP64 && precision != FFTMECH_MIXED) return FFTMECH_ERR_INVALID_ARG;
  if (grid->dim != 2 && grid->dim != 3) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (!(grid->h > 0) || !(grid->h_diff > 0)) return FFTMECH_ERR_INVALID_ARG;
  if (!factor_ok(grid->n[0]) || !factor_ok(grid->n[1]) || grid->n[0] < 2)
    return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (grid->dim == 3 && (!factor_ok(grid->n[2]) || grid->n[1] < 2 || grid->n[2] < 2))
    return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (!(mat->E_solid > 0) || !(mat->E_pore > 0) || !(mat->nu_solid < 0.5) || !(mat->nu_pore < 0.5) ||
      !(mat->nu_solid > -1) || !(mat->nu_pore > -1) || !(mat->D_solid > 0) || !(mat->D_pore > 0) ||
      !(mat->Gc > 0) || !(mat->l0 > 0) || !(mat->kappa >= 0))
    return FFTMECH_ERR_INVALID_ARG;
  if (!(opts->tol >= 0) || opts->max_iter < 0 || opts->launch_mode < 0 || opts->launch_mode > 1)
    return FFTMECH_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return FFTMECH_ERR_CUDA;
  }
  fftmech_ctx* ctx = new (std::nothrow) fftmech_ctx();
  if (!ctx) return FFTMECH_ERR_OOM;
  ctx->dim = grid->dim;
  ctx->nx = grid->n[0];
  ctx->ny = grid->n[1];
  ctx->nz = grid->dim == 3 ? grid->n[2] : 1;
  ctx->N = (long long)ctx->nx * ctx->ny * ctx->nz;
  ctx->B = batch;
  ctx->h = grid->h;
  ctx->h_diff = grid->h_diff;
  ctx->mat = *mat;
  ctx->prec = precision;
  ctx->opts = *opts;
  if (ctx->opts.check_every <= 0) ctx->opts.check_every = 16;
  auto fail = [&](fftmech_status s) {
    fftmech_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
  ctx->nsm = prop.multiProcessorCount;
  ctx->optin = prop.sharedMemPerBlockOptin;
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(FFTMECH_ERR_CUDA);
    ctx->own_stream = true;
  }
  const bool three = grid->dim == 3;
  const bool fp64 = precision == FFTMECH_FP64;
  if (make_plan(ctx->nx, ctx->px) != cudaSuccess || make_plan(ctx->ny, ctx->py) != cudaSuccess ||
      (three && make_plan(ctx->nz, ctx->pz) != cudaSuccess))
    return fail(FFTMECH_ERR_OOM);
  bool shp;
  if (three)
    shp = fp64 ? choose_shape3<double>(ctx->px, ctx->py, ctx->pz, ctx->nsm, ctx->optin, batch, ctx->shape3)
               : choose_shape3<float>(ctx->px, ctx->py, ctx->pz, ctx->nsm, ctx->optin, batch, ctx->shape3);
  else
    shp = fp64 ? choose_shape<double>(ctx->px, ctx->py, ctx->nsm, ctx->optin, ctx->shape, batch)
               : choose_shape<float>(ctx->px, ctx->py, ctx->nsm, ctx->optin, ctx->shape, batch);
  if (shp) {
    const int spec3 = three ? (int)nxs_of(ctx->nx, 3) : ctx->nx;
    shp = fp64 ? choose_line_shape<double>(ctx->px, ctx->ny * ctx->nz, grid->dim, spec3, ctx->nsm, ctx->optin,
                                           batch, ctx->lshape)
               : choose_line_shape<float>(ctx->px, ctx->ny * ctx->nz, grid->dim, spec3, ctx->nsm, ctx->optin,
                                          batch, ctx->lshape);
    ctx->lshape.sst = three ? ctx->shape3.sst : ctx->N;
    choose_sten_shape(ctx->nx, ctx->ny, ctx->nz, grid->dim, ctx->nsm, batch, ctx->sshape);
  }
  if (!shp) return fail(FFTMECH_ERR_UNSUPPORTED_SIZE);
  ctx->shape.batch = batch;
  const size_t es = fp64 ? 8 : 4;
  const size_t NB = (size_t)ctx->N * batch;
  const size_t nd = (size_t)grid->dim;  // displacement components
  // spectral buffer: 2D one packed complex field; 3D the rows of Shape3
  const size_t s_complex = three ? (size_t)ctx->shape3.sst * batch : NB;
  // reduction partials: per problem, one slot group per block of the widest launch
  size_t widest;
  if (three) {
    const Shape3& t = ctx->shape3;
    widest = (size_t)ctx->ny * ((nxs_of(ctx->nx, 3) + t.cw_z - 1) / t.cw_z);  // z-pass blocks
  } else {
    widest = (ctx->nx + ctx->shape.cols - 1) / ctx->shape.cols;  // column strips
  }
  {
    const StenShape& t = ctx->sshape;
    size_t tiles = (size_t)((ctx->nx + t.tx - 1) / t.tx) * ((ctx->ny + t.ty - 1) / t.ty);
    if (three) tiles *= (size_t)((ctx->nz + t.zc - 1) / t.zc);
    widest = std::max(widest, tiles);
  }
  const size_t post_blocks = batch > 1 ? 512 : 4096;
  const size_t slots = (size_t)batch * std::max(widest, post_blocks) * 16;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) ok = false;
  };
  alloc(&ctx->q, nd * NB * es);
  alloc(&ctx->r, nd * NB * es);
  alloc(&ctx->p[0], nd * NB * es);
  alloc(&ctx->p[1], nd * NB * es);
  alloc(&ctx->S, 2 * s_complex * es);
  alloc(&ctx->g, NB * es);
  if (!fp64) {
    alloc((void**)&ctx->uh, nd * NB * sizeof(float));
    alloc((void**)&ctx->ul, nd * NB * sizeof(float));
  }
  alloc((void**)&ctx->phi, NB * 8);
  alloc((void**)&ctx->Hd, NB * 8);
  alloc((void**)&ctx->cn, NB * 8);
  alloc(&ctx->lamx, ctx->nx * es);
  alloc(&ctx->lamy, ctx->ny * es);
  if (three) {
    alloc(&ctx->lamz, ctx->nz * es);
    alloc(&ctx->lamc3, (size_t)nxs_of(ctx->nx, 3) * es);
    alloc(&ctx->wcol3, (size_t)nxs_of(ctx->nx, 3) * es);
    alloc(&ctx->lamc1, (size_t)nxs_of(ctx->nx, 1) * es);
    alloc(&ctx->wcol1, (size_t)nxs_of(ctx->nx, 1) * es);
  }
  alloc((void**)&ctx->partials, slots * 8);
  if (!three) alloc((void**)&ctx->partials_col, (size_t)batch * ctx->nx * 8);
  alloc((void**)&ctx->results, (size_t)kResultsPerProblem * batch * 8);
  alloc((void**)&ctx->m0b, (size_t)batch * 8);
  alloc((void**)&ctx->m1b, (size_t)batch * 8);
  alloc((void**)&ctx->mode, (size_t)batch * sizeof(int));
  alloc((void**)&ctx->sc, sizeof(SolverScalars) * batch);
  if (!ok) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_sc, sizeof(SolverScalars) * batch) != cudaSuccess) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_results, (size_t)kResultsPerProblem * batch * 8) != cudaSuccess)
    return fail(FFTMECH_ERR_OOM);
  ctx->h_mode = new (std::nothrow) int[batch];
  if (!ctx->h_mode) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_mode_ring, sizeof(int) * batch * fftmech_ctx::kModeSlots) != cudaSuccess)
    return fail(FFTMECH_ERR_OOM);
  for (int k = 0; k < fftmech_ctx::kModeSlots; ++k)
    if (cudaEventCreateWithFlags(&ctx->mode_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(FFTMECH_ERR_CUDA);
  if (cudaEventCreate(&ctx->solve_ev[0]) != cudaSuccess || cudaEventCreate(&ctx->solve_ev[1]) != cudaSuccess)
    return fail(FFTMECH_ERR_CUDA);
  fftmech_status rc = fp64 ? fill_lam<double>(ctx) : fill_lam<float>(ctx);
  if (rc != FFTMECH_OK) return fail(rc);
  *out = ctx;
  return FFTMECH_OK;
}

fftmech_status fftmech_create(fftmech_ctx** out, const fftmech_grid* grid,
                              const fftmech_materials* mat, fftmech_precision precision,
                              const fftmech_solver_opts* opts, void* stream) {
  return fftmech_create_batched(out, grid, 1, mat, precision, opts, stream);
}

fftmech_status fftmech_destroy(fftmech_ctx* ctx) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  void* bufs[] = {ctx->r, ctx->q, ctx->p[0], ctx->p[1], ctx->S, ctx->g, ctx->uh, ctx->ul, ctx->phi, ctx->Hd,
                  ctx->cn, ctx->lamx, ctx->lamy, ctx->lamz, ctx->lamc3, ctx->lamc1, ctx->wcol3, ctx->wcol1,
                  ctx->partials, ctx->partials_col, ctx->results, ctx->m0b, ctx->m1b, ctx->mode, ctx->sc};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < ST_COUNT; ++i)
    if (ctx->stage[i].dev) cudaFree(ctx->stage[i].dev);
  if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
  if (ctx->h_results) cudaFreeHost(ctx->h_results);
  delete[] ctx->h_mode;
  if (ctx->h_mode_ring) cudaFreeHost(ctx->h_mode_ring);
  for (cudaEvent_t e : ctx->mode_ev)
    if (e) cudaEventDestroy(e);
  for (auto& pe : ctx->pending) { ctx->ev_free.push_back(pe.a); ctx->ev_free.push_back(pe.b); }
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->solve_ev)
    if (e) cudaEventDestroy(e);
  free_plan(ctx->px);
  free_plan(ctx->py);
  free_plan(ctx->pz);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FFTMECH_OK;
}

fftmech_status fftmech_set_solver_opts(fftmech_ctx* ctx, const fftmech_solver_opts* opts) {
  if (!ctx || !opts) return FFTMECH_ERR_INVALID_ARG;
  if (!(opts->tol >= 0) || opts->max_iter < 0 || opts->launch_mode < 0 || opts->launch_mode > 1)
    return FFTMECH_ERR_INVALID_ARG;
  ctx->opts = *opts;
  if (ctx->opts.check_every <= 0) ctx->opts.check_every = 16;
  return FFTMECH_OK;
}

int fftmech_batch_size(const fftmech_ctx* ctx) { return ctx ? ctx->B : 0; }

fftmech_status fftmech_equilibrium_solve(fftmech_ctx* ctx, const uint8_t* phase, const void* eig,
                                         const double* damage, const double eps_mac[6], double* u,
                                         void* strain, void* stress, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !eps_mac || !u || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(fftmech_solve_info) * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  void *dphase, *deig, *ddmg, *du, *dstrain, *dstress;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &ddmg)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_U, u, (size_t)ctx->dim * N * 8, true, &du)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRAIN, strain, nv * N * es, false, &dstrain)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRESS, stress, nv * N * es, false, &dstress)) != FFTMECH_OK) return rc;
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = equilibrium_impl<double>(ctx, (const uint8_t*)dphase, (const double*)deig, (const double*)ddmg,
                                 eps_mac, (double*)du, (double*)dstrain, (double*)dstress, info, 1);
  else
    s = equilibrium_impl<float>(ctx, (const uint8_t*)dphase, (const float*)deig, (const double*)ddmg,
                                eps_mac, (double*)du, (float*)dstrain, (float*)dstress, info, 1);
  if (is_hard_error(s)) return s;
  if ((rc = stage_out(ctx, u, du, (size_t)ctx->dim * N * 8)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, strain, dstrain, nv * N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, stress, dstress, nv * N * es)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

fftmech_status fftmech_diffusion_step(fftmech_ctx* ctx, const uint8_t* phase, int mode,
                                      const double grad_c_mac[3], double c_macro, double dt,
                                      const uint8_t* dirichlet_mask, double dirichlet_value,
                                      double* c, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !c || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (mode != FFTMECH_DIFF_HOMOGENISE && mode != FFTMECH_DIFF_TRANSIENT)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "diffusion mode %d", mode);
  if (mode == FFTMECH_DIFF_HOMOGENISE && !grad_c_mac)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "grad_c_mac is required");
  std::memset(info, 0, sizeof(fftmech_solve_info) * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B;
  void *dphase, *dc, *dmask = nullptr;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_C, c, N * 8, mode == FFTMECH_DIFF_TRANSIENT, &dc)) != FFTMECH_OK) return rc;
  if (mode == FFTMECH_DIFF_TRANSIENT &&
      (rc = stage_in(ctx, ST_MASK, dirichlet_mask, N, true, &dmask)) != FFTMECH_OK)
    return rc;
  const double zero[3] = {0, 0, 0};
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = diffusion_impl<double>(ctx, (const uint8_t*)dphase, mode, grad_c_mac ? grad_c_mac : zero, c_macro, dt,
                               (const uint8_t*)dmask, dirichlet_value, (double*)dc, info, 1);
  else
    s = diffusion_impl<float>(ctx, (const uint8_t*)dphase, mode, grad_c_mac ? grad_c_mac : zero, c_macro, dt,
                              (const uint8_t*)dmask, dirichlet_value, (double*)dc, info, 1);
  if (is_hard_error(s)) return s;
  if ((rc = stage_out(ctx, c, dc, N * 8)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

fftmech_status fftmech_phasefield_solve(fftmech_ctx* ctx, const void* strain, const void* eig,
                                        const uint8_t* phase, void* H, double* damage,
                                        fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!strain || !phase || !H || !damage || !info)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(fftmech_solve_info) * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  void *dstrain, *deig, *dphase, *dH, *dd;
  if ((rc = stage_in(ctx, ST_STRAIN, strain, nv * N * es, true, &dstrain)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_H, H, N * es, true, &dH)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &dd)) != FFTMECH_OK) return rc;
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = phasefield_impl<double>(ctx, (const double*)dstrain, (const double*)deig, (const uint8_t*)dphase,
                                (double*)dH, (double*)dd, info, 1);
  else
    s = phasefield_impl<float>(ctx, (const float*)dstrain, (const float*)deig, (const uint8_t*)dphase,
                               (float*)dH, (double*)dd, info, 1);
  if (is_hard_error(s)) return s;
  if ((rc = stage_out(ctx, H, dH, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, damage, dd, N * 8)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

fftmech_status fftmech_staggered_step(fftmech_ctx* ctx, fftmech_state* state,
                                      const fftmech_step_params* prm, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!state || !prm || !info || !state->phase || !state->c || !state->eig || !state->u ||
      !state->strain || !state->stress || !state->H || !state->damage)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (prm->eig_mode == FFTMECH_EIG_PRESCRIBED && !prm->eig_field)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "eig_field is required for PRESCRIBED");
  std::memset(info, 0, sizeof(fftmech_solve_info) * 3 * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  cudaStream_t st = ctx->stream;
  void *dphase, *dc, *dcppt, *deig, *du, *dstrain, *dstress, *dH, *dd, *dmask = nullptr, *deigf = nullptr;
  if ((rc = stage_in(ctx, ST_PHASE, state->phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_C, state->c, N * 8, true, &dc)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_CPPT, state->c_ppt, N * es, true, &dcppt)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, state->eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_U, state->u, (size_t)ctx->dim * N * 8, true, &du)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRAIN, state->strain, nv * N * es, true, &dstrain)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRESS, state->stress, nv * N * es, true, &dstress)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_H, state->H, N * es, true, &dH)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_DAMAGE, state->damage, N * 8, true, &dd)) != FFTMECH_OK) return rc;
  if (prm->diffusion_mode == FFTMECH_DIFF_TRANSIENT &&
      (rc = stage_in(ctx, ST_MASK, prm->dirichlet_mask, N, true, &dmask)) != FFTMECH_OK)
    return rc;
  if (prm->eig_mode == FFTMECH_EIG_PRESCRIBED &&
      (rc = stage_in(ctx, ST_EIGFIELD, prm->eig_field, N * es, true, &deigf)) != FFTMECH_OK)
    return rc;
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  fftmech_status worst = FFTMECH_OK;
  auto track = [&](fftmech_status s) {
    if (s != FFTMECH_OK && worst == FFTMECH_OK) worst = s;
  };
  // 1. diffusion of chemical species
  if (prm->diffusion_mode != FFTMECH_DIFF_NONE) {
    fftmech_status s = fp64
        ? diffusion_impl<double>(ctx, (const uint8_t*)dphase, prm->diffusion_mode, prm->grad_c_mac,
                                 prm->c_macro, prm->dt, (const uint8_t*)dmask, prm->dirichlet_value,
                                 (double*)dc, info + 0, 3)
        : diffusion_impl<float>(ctx, (const uint8_t*)dphase, prm->diffusion_mode, prm->grad_c_mac,
                                prm->c_macro, prm->dt, (const uint8_t*)dmask, prm->dirichlet_value,
                                (double*)dc, info + 0, 3);
    if (is_hard_error(s)) return s;
    track(s);
  }
  // 2. precipitation and eigenstrain
  if (prm->eig_mode == FFTMECH_EIG_FROM_PRECIPITATE) {
    ProfScope _ps(ctx, FFTMECH_K_OTHER);
    if (fp64)
      CK(launch_precipitate<double>(N, (const uint8_t*)dphase, (const double*)dc, ctx->mat.S_sol,
                                    ctx->mat.M_ppt, (double*)dcppt, (double*)deig, st));
    else
      CK(launch_precipitate<float>(N, (const uint8_t*)dphase, (const double*)dc, ctx->mat.S_sol,
                                   ctx->mat.M_ppt, (float*)dcppt, (float*)deig, st));
  } else {
    ProfScope _ps(ctx, FFTMECH_K_OTHER);
    if (fp64)
      CK(launch_scale_copy<double>(N, (const double*)deigf, prm->eig_scale, (double*)deig, st));
    else
      CK(launch_scale_copy<float>(N, (const float*)deigf, prm->eig_scale, (float*)deig, st));
  }
  // 3. equilibrium with the stiffness degraded by the current damage
  {
    fftmech_status s = fp64
        ? equilibrium_impl<double>(ctx, (const uint8_t*)dphase, (const double*)deig, (const double*)dd,
                                   prm->eps_mac, (double*)du, (double*)dstrain, (double*)dstress, info + 1, 3)
        : equilibrium_impl<float>(ctx, (const uint8_t*)dphase, (const float*)deig, (const double*)dd,
                                  prm->eps_mac, (double*)du, (float*)dstrain, (float*)dstress, info + 1, 3);
    if (is_hard_error(s)) return s;
    track(s);
  }
  // 4. history and phase field
  {
    fftmech_status s = fp64
        ? phasefield_impl<double>(ctx, (const double*)dstrain, (const double*)deig, (const uint8_t*)dphase,
                                  (double*)dH, (double*)dd, info + 2, 3)
        : phasefield_impl<float>(ctx, (const float*)dstrain, (const float*)deig, (const uint8_t*)dphase,
                                 (float*)dH, (double*)dd, info + 2, 3);
    if (is_hard_error(s)) return s;
    track(s);
  }
  if ((rc = stage_out(ctx, state->c, dc, N * 8)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->c_ppt, dcppt, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->eig, deig, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->u, du, (size_t)ctx->dim * N * 8)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->strain, dstrain, nv * N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->stress, dstress, nv * N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->H, dH, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->damage, dd, N * 8)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(st));
  return worst;
}

fftmech_status fftmech_staggered_step_many(fftmech_ctx* const* ctxs, int n, fftmech_state* const* states,
                                           const fftmech_step_params* const* params,
                                           fftmech_solve_info* const* infos) {
  if (!ctxs || !states || !params || !infos || n < 0) return FFTMECH_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !states[i] || !params[i] || !infos[i]) return FFTMECH_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream) return FFTMECH_ERR_INVALID_ARG;
  }
  std::vector<fftmech_status> rc(n, FFTMECH_OK);
  std::vector<std::thread> workers;
  workers.reserve(n);
  for (int i = 0; i < n; ++i)
    workers.emplace_back([&, i]() { rc[i] = fftmech_staggered_step(ctxs[i], states[i], params[i], infos[i]); });
  for (auto& w : workers) w.join();
  for (int i = 0; i < n; ++i)
    if (is_hard_error(rc[i])) return rc[i];
  for (int i = 0; i < n; ++i)
    if (rc[i] != FFTMECH_OK) return rc[i];
  return FFTMECH_OK;
}

fftmech_status fftmech_profile_enable(fftmech_ctx* ctx, int enable) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  prof_flush(ctx);
  ctx->prof = enable != 0;
  for (int k = 0; k < FFTMECH_K_COUNT; ++k) {
    ctx->launches[k] = 0;
    ctx->prof_ms[k] = 0.0;
  }
  return FFTMECH_OK;
}

fftmech_status fftmech_profile_read(fftmech_ctx* ctx, int kclass, long long* launches,
                                    double* total_ms) {
  if (!ctx || !launches || !total_ms || kclass < 0 || kclass > FFTMECH_K_COUNT)
    return FFTMECH_ERR_INVALID_ARG;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  prof_flush(ctx);
  if (kclass == FFTMECH_K_COUNT) {
    long long n = 0;
    double ms = 0;
    for (int k = 0; k < FFTMECH_K_COUNT; ++k) { n += ctx->launches[k]; ms += ctx->prof_ms[k]; }
    *launches = n;
    *total_ms = ms;
  } else {
    *launches = ctx->launches[kclass];
    *total_ms = ctx->prof_ms[kclass];
  }
  return FFTMECH_OK;
}

fftmech_status fftmech_fft(int ndim, const int n[3], int precision, int inverse, void* data,
                           void* stream) {
  fftmech_ctx* ctx = nullptr;  // for CK's error path (no message storage)
  if (!n || !data || (ndim != 1 && ndim != 2)) return FFTMECH_ERR_INVALID_ARG;
  if (precision != FFTMECH_FP64 && precision != FFTMECH_MIXED) return FFTMECH_ERR_INVALID_ARG;
  const int nx = n[0], ny = ndim == 2 ? n[1] : 1;
  if (!factor_ok(nx) || !factor_ok(ny) || nx < 2) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (!is_device_ptr(data)) return FFTMECH_ERR_INVALID_ARG;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  HostPlan px, py;
  cudaError_t e1 = make_plan(nx, px), e2 = make_plan(ny, py);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    free_plan(px);
    free_plan(py);
    return FFTMECH_ERR_OOM;
  }
  const bool fp64 = precision == FFTMECH_FP64;
  fftmech_status rc = FFTMECH_OK;
  Shape2 sh{};
  const bool shp = fp64 ? choose_shape_fft<double>(px, py, prop.multiProcessorCount, prop.sharedMemPerBlockOptin, sh)
                        : choose_shape_fft<float>(px, py, prop.multiProcessorCount, prop.sharedMemPerBlockOptin, sh);
  if (!shp) {
    rc = FFTMECH_ERR_UNSUPPORTED_SIZE;
  } else {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (fp64) {
      Spec<double> sp{};
      e = launch_rowfft_f<double>(px.fam, nx, ny, (cx<double>*)data, dev_plan<double>(px), inverse, sh, st);
      if (e == cudaSuccess && ny > 1)
        e = launch_colpass_f<double>(py.fam, nx, ny, (cx<double>*)data, dev_plan<double>(py), sp, sh, COL_PLAIN,
                                   inverse, nullptr, nullptr, nullptr, st);
    } else {
      Spec<float> sp{};
      e = launch_rowfft_f<float>(px.fam, nx, ny, (cx<float>*)data, dev_plan<float>(px), inverse, sh, st);
      if (e == cudaSuccess && ny > 1)
        e = launch_colpass_f<float>(py.fam, nx, ny, (cx<float>*)data, dev_plan<float>(py), sp, sh, COL_PLAIN,
                                  inverse, nullptr, nullptr, nullptr, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = FFTMECH_ERR_CUDA;
  }
  free_plan(px);
  free_plan(py);
  return rc;
}

}  // extern "C"
