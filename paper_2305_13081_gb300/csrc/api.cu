// C ABI of libfftmech: contexts, FFT plans, workspace, the PCG driver and the
// entry points declared in include/fftmech.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fftmech.h"
#include "fftmech_internal.cuh"
#include "host_plan.cuh"

using namespace fftmech;

namespace {

constexpr int kMaxBlocks = 8192;     // upper bound on reduction partials per launch
constexpr int kPartialSlots = 16;    // doubles per block in `partials`

// ---------------------------------------------------------------- plans
// Device twiddles for a context (FP64 values from the host, also rounded to
// float).
cudaError_t make_plan(int n, HostPlan& p) {
  factor_plan(n, p);
  const int nt = std::max(twiddle_count(p), 1);
  std::vector<cx<double>> hd(nt);
  std::vector<cx<float>> hf(nt);
  fill_twiddles(p, hd.data());
  for (int i = 0; i < nt; ++i) {
    hf[i].re = (float)hd[i].re;
    hf[i].im = (float)hd[i].im;
  }
  cudaError_t e = cudaMalloc(&p.tw_f, nt * sizeof(cx<float>));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p.tw_d, nt * sizeof(cx<double>));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(p.tw_f, hf.data(), nt * sizeof(cx<float>), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(p.tw_d, hd.data(), nt * sizeof(cx<double>), cudaMemcpyHostToDevice);
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
  long long N = 0;
  double h = 1, h_diff = 1;
  fftmech_materials mat{};
  fftmech_precision prec = FFTMECH_FP64;
  fftmech_solver_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int nsm = 0;
  size_t optin = 0;
  HostPlan px, py;
  Shape2 shape_f{}, shape_d{};
  // workspace
  void* r = nullptr;
  void* p[2] = {nullptr, nullptr};
  void* S = nullptr;
  void* g = nullptr;
  float* uh = nullptr;  // MIXED iterate, high part (2 N)
  float* ul = nullptr;  // MIXED iterate, low part (2 N)
  double* phi = nullptr;
  double* Hd = nullptr;
  double* cn = nullptr;
  void* lamx = nullptr;
  void* lamy = nullptr;
  double* partials = nullptr;
  double* results = nullptr;
  SolverScalars* sc = nullptr;
  unsigned int* cnt = nullptr;
  SolverScalars* h_sc = nullptr;   // pinned
  double* h_results = nullptr;     // pinned
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

void lame(double E, double nu, double& lam, double& mu) {
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  mu = E / (2.0 * (1.0 + nu));
}

void fill_info_defaults(fftmech_solve_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
}

// ---------------------------------------------------------------- PCG driver
template <typename T>
struct Solve {
  int iters = 0;
  int status = FFTMECH_OK;
  double rel = 0, true_rel = 0;
};

template <typename T, int D>
fftmech_status run_pcg(fftmech_ctx* ctx, const Op2<T>& op, double* u, double m0, double m1,
                       Solve<T>& out) {
  cudaStream_t st = ctx->stream;
  const Shape2& sh = sizeof(T) == 4 ? ctx->shape_f : ctx->shape_d;
  FftPlanDev<T> px = dev_plan<T>(ctx->px), py = dev_plan<T>(ctx->py);
  Spec2<T> sp;
  sp.lamx = (const T*)ctx->lamx;
  sp.lamy = (const T*)ctx->lamy;
  sp.m0 = m0;
  sp.m1 = m1;
  sp.invN = 1.0 / (double)ctx->N;
  SolverScalars h{};
  h.tol2 = ctx->opts.tol * ctx->opts.tol;
  h.max_iter = ctx->opts.max_iter;
  CK(cudaMemcpyAsync(ctx->sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  T* pbuf[2] = {(T*)ctx->p[0], (T*)ctx->p[1]};
  Vec2<T> v;
  v.u = u;
  v.uh = ctx->uh;
  v.ul = ctx->ul;
  const long long nU = (long long)D * ctx->N;
  if (sizeof(T) == 4) CK(launch_df_split(nU, u, ctx->uh, ctx->ul, st));
  v.r = (T*)ctx->r;
  v.p_in = pbuf[0];
  v.p_out = pbuf[1];
  v.S = (cx<T>*)ctx->S;
  v.partials = ctx->partials;
  v.sc = ctx->sc;
  const int nx = ctx->nx, ny = ctx->ny;
#define FFTMECH_LAUNCH(KC, CALL) \
  do {                           \
    ProfScope _ps(ctx, KC);      \
    CK(CALL);                    \
  } while (0)
  FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, (launch_residual_f<T, D>(ctx->px.fam, op, v, px, sh, 1, st)));
  FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_NORM, 0, ctx->partials, ctx->sc, st));
  FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, (launch_residual_f<T, D>(ctx->px.fam, op, v, px, sh, 0, st)));
  FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_INIT, 0, ctx->partials, ctx->sc, st));
  CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  prof_flush(ctx);
  if (ctx->h_sc->rz0 == 0.0 && ctx->h_sc->rz > 0.0) {
    // zero right-hand side: the solution is zero (outside Dirichlet voxels)
    if (op.mask) {
      return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "zero right-hand side with a Dirichlet mask");
    }
    CK(cudaMemsetAsync(u, 0, sizeof(double) * D * ctx->N, st));
    out.iters = 0;
    out.status = FFTMECH_OK;
    out.rel = out.true_rel = 0.0;
    return FFTMECH_OK;
  }
  const int check = std::max(1, ctx->opts.check_every);
  const bool reliable = (sizeof(T) == 4) && ctx->opts.replace_residual != 0;
  double rz_rep = ctx->h_sc->rz;  // r.M^-1 r right after the last (true) residual
  bool pending = false;
  int pi = 0;
  int it = 0;
  bool done = ctx->h_sc->done != 0;
  for (int restart = 0;; ++restart) {
    while (!done && it < ctx->opts.max_iter) {
      Vec2<T> va = v;
      va.p_in = pbuf[pi];
      va.p_out = pbuf[1 - pi];
      FFTMECH_LAUNCH(FFTMECH_K_DIRECTION, (launch_direction_f<T, D>(ctx->px.fam, op, va, px, sh, st)));
      Vec2<T> vb = v;
      vb.p_in = pbuf[1 - pi];
      const bool replace = pending;
      pending = false;
      if (replace) {
        // reliable update: u += alpha p only, then the FP64 true residual
        FFTMECH_LAUNCH(FFTMECH_K_UPDATE, (launch_update_f<T, D>(ctx->px.fam, op, vb, px, sh, 1, st)));
        FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, (launch_residual_f<T, D>(ctx->px.fam, op, v, px, sh, 0, st)));
        FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_TRUE, 0, ctx->partials, ctx->sc, st));
      } else {
        FFTMECH_LAUNCH(FFTMECH_K_UPDATE, (launch_update_f<T, D>(ctx->px.fam, op, vb, px, sh, 0, st)));
        FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_ITER, 0, ctx->partials, ctx->sc, st));
      }
      pi = 1 - pi;
      ++it;
      if (it % check == 0 || it >= ctx->opts.max_iter || replace) {
        CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        prof_flush(ctx);
        done = ctx->h_sc->done != 0;
        if (replace) rz_rep = ctx->h_sc->rz_true;
        else if (reliable && ctx->h_sc->rz < 1e-2 * rz_rep) pending = true;
      }
    }
    // FP64 true residual of the iterate
    FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, (launch_residual_f<T, D>(ctx->px.fam, op, v, px, sh, 0, st)));
    FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_TRUENORM, 0, ctx->partials, ctx->sc, st));
    CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prof_flush(ctx);
    const SolverScalars& q = *ctx->h_sc;
    const bool gate = reliable && q.status == FFTMECH_OK && restart < 3 && q.iter < ctx->opts.max_iter &&
                      q.rz_true > 4.0 * q.tol2 * q.rz0;
    if (!gate) break;
    // the float recursion met tol but the true residual did not: continue
    // from the true residual with a fresh direction
    const int zero = 0;
    CK(cudaMemcpyAsync(&ctx->sc->done, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    FFTMECH_LAUNCH(FFTMECH_K_RESIDUAL, (launch_residual_f<T, D>(ctx->px.fam, op, v, px, sh, 0, st)));
    FFTMECH_LAUNCH(FFTMECH_K_COLUMN, launch_colpass_f<T>(ctx->py.fam, nx, ny, v.S, py, sp, sh, COL_RESTART, 0, ctx->partials, ctx->sc, st));
    CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prof_flush(ctx);
    done = ctx->h_sc->done != 0;
    rz_rep = ctx->h_sc->rz;
    pending = false;
  }
  if (sizeof(T) == 4) {
    CK(launch_df_merge(nU, ctx->uh, ctx->ul, u, st));
  }
  const SolverScalars& f = *ctx->h_sc;
  out.iters = f.iter;
  out.status = f.done ? f.status : FFTMECH_ERR_NOT_CONVERGED;
  out.rel = f.rz0 > 0 ? std::sqrt(std::max(f.rz, 0.0) / f.rz0) : 0.0;
  out.true_rel = f.rz0 > 0 ? std::sqrt(std::max(f.rz_true, 0.0) / f.rz0) : 0.0;
  return FFTMECH_OK;
}

template <typename T>
void base_op(const fftmech_ctx* ctx, Op2<T>& op, const uint8_t* phase) {
  std::memset(&op, 0, sizeof(op));
  op.nx = ctx->nx;
  op.ny = ctx->ny;
  op.h = ctx->h;
  op.phase = phase;
  lame(ctx->mat.E_pore, ctx->mat.nu_pore, op.lam[0], op.mu[0]);
  lame(ctx->mat.E_solid, ctx->mat.nu_solid, op.lam[1], op.mu[1]);
  op.src_scale = 1.0;
}

fftmech_status read_results(fftmech_ctx* ctx, int n) {
  CK(cudaMemcpyAsync(ctx->h_results, ctx->results, sizeof(double) * n, cudaMemcpyDeviceToHost,
                     ctx->stream));
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

void copy_solve(const Solve<float>& s, fftmech_solve_info* info) {
  info->status = s.status; info->iters = s.iters; info->rel_res = s.rel; info->true_rel_res = s.true_rel;
}
void copy_solve(const Solve<double>& s, fftmech_solve_info* info) {
  info->status = s.status; info->iters = s.iters; info->rel_res = s.rel; info->true_rel_res = s.true_rel;
}

// ---------------------------------------------------------------- solves
template <typename T>
fftmech_status equilibrium_impl(fftmech_ctx* ctx, const uint8_t* phase, const T* eig,
                                const double* damage, const double* eps_mac, double* u, T* strain,
                                T* stress, fftmech_solve_info* info) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc0 = solve_timer_start(ctx);
  if (rc0 != FFTMECH_OK) return rc0;
  Op2<T> op;
  base_op<T>(ctx, op, phase);
  op.eig = eig;
  op.E[0] = eps_mac[0];
  op.E[1] = eps_mac[1];
  op.E[2] = eps_mac[2];
  if (damage) {
    { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_degradation<T>(ctx->N, damage, ctx->mat.kappa, (T*)ctx->g, st)); }
    op.g = (const T*)ctx->g;
  }
  Solve<T> s;
  fftmech_status rc = run_pcg<T, 2>(ctx, op, u, 0.0, 1.0 / (ctx->h * ctx->h), s);
  if (rc != FFTMECH_OK) return rc;
  { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_el_output<T>(op, u, strain, stress, ctx->partials, ctx->results, &ctx->sc->cnt[2], st)); }
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  rc = read_results(ctx, 7);
  if (rc != FFTMECH_OK) return rc;
  info->device_ms = solve_timer_ms(ctx);
  const double* R = ctx->h_results;
  const double N = (double)ctx->N;
  copy_solve(s, info);
  for (int k = 0; k < 3; ++k) {
    info->mean_stress[k] = R[k] / N;
    info->mean_strain[k] = R[3 + k] / N;
  }
  info->elastic_energy = R[6] * ctx->h * ctx->h;
  return (fftmech_status)s.status;
}

template <typename T>
fftmech_status diffusion_impl(fftmech_ctx* ctx, const uint8_t* phase, int mode,
                              const double* grad_c_mac, double c_macro, double dt,
                              const uint8_t* mask, double cD, double* c,
                              fftmech_solve_info* info) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc0 = solve_timer_start(ctx);
  if (rc0 != FFTMECH_OK) return rc0;
  Op2<T> op;
  base_op<T>(ctx, op, phase);
  op.h = ctx->h_diff;
  op.kap[0] = ctx->mat.D_pore;
  op.kap[1] = ctx->mat.D_solid;
  const double ih2 = 1.0 / (ctx->h_diff * ctx->h_diff);
  Solve<T> s;
  fftmech_status rc;
  if (mode == FFTMECH_DIFF_HOMOGENISE) {
    op.G[0] = grad_c_mac[0];
    op.G[1] = grad_c_mac[1];
    rc = run_pcg<T, 1>(ctx, op, ctx->phi, 0.0, ih2, s);
    if (rc != FFTMECH_OK) return rc;
    { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_diff_stats<T>(op, ctx->phi, ctx->h_diff, c_macro, ctx->partials, ctx->results,
                            &ctx->sc->cnt[2], st)); }
    { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_diff_write_c(ctx->nx, ctx->ny, phase, ctx->phi, ctx->h_diff, op.G[0], op.G[1],
                           ctx->results, c, st)); }
    if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
    rc = read_results(ctx, 5);
    if (rc != FFTMECH_OK) return rc;
    info->device_ms = solve_timer_ms(ctx);
    copy_solve(s, info);
    info->mean_flux[0] = ctx->h_results[2];
    info->mean_flux[1] = ctx->h_results[3];
    info->porosity = ctx->h_results[4];
    info->mean_c = c_macro;
    return (fftmech_status)s.status;
  }
  // TRANSIENT (backward Euler, not in the paper)
  if (!(dt > 0)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt must be > 0 for TRANSIENT");
  { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_pf_stats(ctx->N, phase, nullptr, ctx->partials, ctx->results, &ctx->sc->cnt[2], st)); }
  rc = read_results(ctx, 3);
  if (rc != FFTMECH_OK) return rc;
  const double eta = 1.0 - ctx->h_results[2] / (double)ctx->N;
  const double Dbar = eta * ctx->mat.D_pore + (1.0 - eta) * ctx->mat.D_solid;
  if (mask) {
    ProfScope _ps(ctx, FFTMECH_K_OTHER);
    CK(launch_set_masked(ctx->N, mask, cD, c, st));
  }
  CK(cudaMemcpyAsync(ctx->cn, c, sizeof(double) * ctx->N, cudaMemcpyDeviceToDevice, st));
  op.c0c = 1.0 / dt;
  op.srcd = ctx->cn;
  op.src_scale = 1.0 / dt;
  op.mask = mask;
  rc = run_pcg<T, 1>(ctx, op, c, 1.0 / dt, Dbar * ih2, s);
  if (rc != FFTMECH_OK) return rc;
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  copy_solve(s, info);
  info->device_ms = solve_timer_ms(ctx);
  info->porosity = eta;
  return (fftmech_status)s.status;
}

template <typename T>
fftmech_status phasefield_impl(fftmech_ctx* ctx, const T* strain, const T* eig,
                               const uint8_t* phase, T* H, double* d, fftmech_solve_info* info) {
  cudaStream_t st = ctx->stream;
  fftmech_status rc0 = solve_timer_start(ctx);
  if (rc0 != FFTMECH_OK) return rc0;
  Op2<T> op;
  base_op<T>(ctx, op, phase);
  { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_history<T>(ctx->N, phase, op.lam[0], op.lam[1], op.mu[0], op.mu[1], strain, eig, H,
                       ctx->Hd, ctx->partials, ctx->results, &ctx->sc->cnt[2], st)); }
  fftmech_status rc = read_results(ctx, 1);
  if (rc != FFTMECH_OK) return rc;
  const double Hbar = ctx->h_results[0] / (double)ctx->N;
  const double a = ctx->mat.Gc / (2.0 * ctx->mat.l0);
  const double b = ctx->mat.Gc * ctx->mat.l0 / 2.0;
  op.kap[0] = op.kap[1] = b;
  op.c0c = a;
  op.c0f = H;
  op.srcd = ctx->Hd;
  op.src_scale = 1.0;
  Solve<T> s;
  rc = run_pcg<T, 1>(ctx, op, d, a + Hbar, b / (ctx->h * ctx->h), s);
  if (rc != FFTMECH_OK) return rc;
  { ProfScope _ps(ctx, FFTMECH_K_OTHER); CK(launch_pf_stats(ctx->N, phase, d, ctx->partials, ctx->results, &ctx->sc->cnt[2], st)); }
  if ((rc = solve_timer_stop(ctx)) != FFTMECH_OK) return rc;
  rc = read_results(ctx, 3);
  if (rc != FFTMECH_OK) return rc;
  info->device_ms = solve_timer_ms(ctx);
  copy_solve(s, info);
  info->total_damage = ctx->h_results[0];
  info->frac_damaged = ctx->h_results[2] > 0 ? ctx->h_results[1] / ctx->h_results[2] : 0.0;
  return (fftmech_status)s.status;
}

fftmech_status check_ctx(fftmech_ctx* ctx) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return set_err(ctx, FFTMECH_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  return FFTMECH_OK;
}

template <typename T>
fftmech_status fill_lam(fftmech_ctx* ctx) {
  std::vector<T> lx(ctx->nx), ly(ctx->ny);
  for (int k = 0; k < ctx->nx; ++k) lx[k] = (T)(2.0 - 2.0 * std::cos(2.0 * M_PI * k / ctx->nx));
  for (int k = 0; k < ctx->ny; ++k) ly[k] = (T)(2.0 - 2.0 * std::cos(2.0 * M_PI * k / ctx->ny));
  CK(cudaMemcpy(ctx->lamx, lx.data(), sizeof(T) * ctx->nx, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->lamy, ly.data(), sizeof(T) * ctx->ny, cudaMemcpyHostToDevice));
  return FFTMECH_OK;
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

fftmech_status fftmech_create(fftmech_ctx** out, const fftmech_grid* grid,
                              const fftmech_materials* mat, fftmech_precision precision,
                              const fftmech_solver_opts* opts, void* stream) {
  if (!out || !grid || !mat || !opts) return FFTMECH_ERR_INVALID_ARG;
  *out = nullptr;
  if (precision != FFTMECH_FP64 && precision != FFTMECH_MIXED) return FFTMECH_ERR_INVALID_ARG;
  if (grid->dim != 2) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (!(grid->h > 0) || !(grid->h_diff > 0)) return FFTMECH_ERR_INVALID_ARG;
  if (!factor_ok(grid->n[0]) || !factor_ok(grid->n[1]) || grid->n[0] < 2)
    return FFTMECH_ERR_UNSUPPORTED_SIZE;
  if (!(mat->E_solid > 0) || !(mat->E_pore > 0) || !(mat->nu_solid < 0.5) || !(mat->nu_pore < 0.5) ||
      !(mat->nu_solid > -1) || !(mat->nu_pore > -1) || !(mat->D_solid > 0) || !(mat->D_pore > 0) ||
      !(mat->Gc > 0) || !(mat->l0 > 0) || !(mat->kappa >= 0))
    return FFTMECH_ERR_INVALID_ARG;
  if (!(opts->tol >= 0) || opts->max_iter < 0) return FFTMECH_ERR_INVALID_ARG;
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
  ctx->nz = 1;
  ctx->N = (long long)ctx->nx * ctx->ny;
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
  if (make_plan(ctx->nx, ctx->px) != cudaSuccess || make_plan(ctx->ny, ctx->py) != cudaSuccess)
    return fail(FFTMECH_ERR_OOM);
  const bool fp64 = precision == FFTMECH_FP64;
  const bool shp = fp64 ? choose_shape<double>(ctx->px, ctx->py, ctx->nsm, ctx->optin, ctx->shape_d)
                        : choose_shape<float>(ctx->px, ctx->py, ctx->nsm, ctx->optin, ctx->shape_f);
  if (!shp) return fail(FFTMECH_ERR_UNSUPPORTED_SIZE);
  const size_t es = fp64 ? 8 : 4;
  const size_t N = (size_t)ctx->N;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) ok = false;
  };
  alloc(&ctx->r, 2 * N * es);
  alloc(&ctx->p[0], 2 * N * es);
  alloc(&ctx->p[1], 2 * N * es);
  alloc(&ctx->S, 2 * N * es);
  alloc(&ctx->g, N * es);
  alloc((void**)&ctx->uh, 2 * N * sizeof(float));
  alloc((void**)&ctx->ul, 2 * N * sizeof(float));
  alloc((void**)&ctx->phi, N * 8);
  alloc((void**)&ctx->Hd, N * 8);
  alloc((void**)&ctx->cn, N * 8);
  alloc(&ctx->lamx, ctx->nx * es);
  alloc(&ctx->lamy, ctx->ny * es);
  alloc((void**)&ctx->partials, (size_t)kMaxBlocks * kPartialSlots * 8);
  alloc((void**)&ctx->results, 64 * 8);
  alloc((void**)&ctx->sc, sizeof(SolverScalars));
  if (!ok) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_sc, sizeof(SolverScalars)) != cudaSuccess) return fail(FFTMECH_ERR_OOM);
  if (cudaEventCreate(&ctx->solve_ev[0]) != cudaSuccess || cudaEventCreate(&ctx->solve_ev[1]) != cudaSuccess)
    return fail(FFTMECH_ERR_CUDA);
  if (cudaMallocHost((void**)&ctx->h_results, 64 * 8) != cudaSuccess) return fail(FFTMECH_ERR_OOM);
  fftmech_status rc = fp64 ? fill_lam<double>(ctx) : fill_lam<float>(ctx);
  if (rc != FFTMECH_OK) return fail(rc);
  *out = ctx;
  return FFTMECH_OK;
}

fftmech_status fftmech_destroy(fftmech_ctx* ctx) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  void* bufs[] = {ctx->r, ctx->p[0], ctx->p[1], ctx->S, ctx->g, ctx->uh, ctx->ul, ctx->phi, ctx->Hd, ctx->cn,
                  ctx->lamx, ctx->lamy, ctx->partials, ctx->results, ctx->sc};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < ST_COUNT; ++i)
    if (ctx->stage[i].dev) cudaFree(ctx->stage[i].dev);
  if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
  for (auto& pe : ctx->pending) { ctx->ev_free.push_back(pe.a); ctx->ev_free.push_back(pe.b); }
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->solve_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->h_results) cudaFreeHost(ctx->h_results);
  free_plan(ctx->px);
  free_plan(ctx->py);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FFTMECH_OK;
}

fftmech_status fftmech_set_solver_opts(fftmech_ctx* ctx, const fftmech_solver_opts* opts) {
  if (!ctx || !opts) return FFTMECH_ERR_INVALID_ARG;
  if (!(opts->tol >= 0) || opts->max_iter < 0) return FFTMECH_ERR_INVALID_ARG;
  ctx->opts = *opts;
  if (ctx->opts.check_every <= 0) ctx->opts.check_every = 16;
  return FFTMECH_OK;
}

fftmech_status fftmech_equilibrium_solve(fftmech_ctx* ctx, const uint8_t* phase, const void* eig,
                                         const double* damage, const double eps_mac[6], double* u,
                                         void* strain, void* stress, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !eps_mac || !u || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  fill_info_defaults(info);
  const size_t N = (size_t)ctx->N, es = esize(ctx), nv = nvoigt(ctx);
  void *dphase, *deig, *ddmg, *du, *dstrain, *dstress;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &ddmg)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_U, u, 2 * N * 8, true, &du)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRAIN, strain, nv * N * es, false, &dstrain)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_STRESS, stress, nv * N * es, false, &dstress)) != FFTMECH_OK) return rc;
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = equilibrium_impl<double>(ctx, (const uint8_t*)dphase, (const double*)deig,
                                 (const double*)ddmg, eps_mac, (double*)du, (double*)dstrain,
                                 (double*)dstress, info);
  else
    s = equilibrium_impl<float>(ctx, (const uint8_t*)dphase, (const float*)deig,
                                (const double*)ddmg, eps_mac, (double*)du, (float*)dstrain,
                                (float*)dstress, info);
  if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
  if ((rc = stage_out(ctx, u, du, 2 * N * 8)) != FFTMECH_OK) return rc;
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
  fill_info_defaults(info);
  const size_t N = (size_t)ctx->N;
  void *dphase, *dc, *dmask = nullptr;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_C, c, N * 8, mode == FFTMECH_DIFF_TRANSIENT, &dc)) != FFTMECH_OK) return rc;
  if (mode == FFTMECH_DIFF_TRANSIENT &&
      (rc = stage_in(ctx, ST_MASK, dirichlet_mask, N, true, &dmask)) != FFTMECH_OK)
    return rc;
  const double zero[3] = {0, 0, 0};
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = diffusion_impl<double>(ctx, (const uint8_t*)dphase, mode, grad_c_mac ? grad_c_mac : zero,
                               c_macro, dt, (const uint8_t*)dmask, dirichlet_value, (double*)dc, info);
  else
    s = diffusion_impl<float>(ctx, (const uint8_t*)dphase, mode, grad_c_mac ? grad_c_mac : zero,
                              c_macro, dt, (const uint8_t*)dmask, dirichlet_value, (double*)dc, info);
  if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
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
  fill_info_defaults(info);
  const size_t N = (size_t)ctx->N, es = esize(ctx), nv = nvoigt(ctx);
  void *dstrain, *deig, *dphase, *dH, *dd;
  if ((rc = stage_in(ctx, ST_STRAIN, strain, nv * N * es, true, &dstrain)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_PHASE, phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_H, H, N * es, true, &dH)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &dd)) != FFTMECH_OK) return rc;
  fftmech_status s;
  if (ctx->prec == FFTMECH_FP64)
    s = phasefield_impl<double>(ctx, (const double*)dstrain, (const double*)deig,
                                (const uint8_t*)dphase, (double*)dH, (double*)dd, info);
  else
    s = phasefield_impl<float>(ctx, (const float*)dstrain, (const float*)deig,
                               (const uint8_t*)dphase, (float*)dH, (double*)dd, info);
  if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
  if ((rc = stage_out(ctx, H, dH, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, damage, dd, N * 8)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

fftmech_status fftmech_staggered_step(fftmech_ctx* ctx, fftmech_state* state,
                                      const fftmech_step_params* prm, fftmech_solve_info info[3]) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!state || !prm || !info || !state->phase || !state->c || !state->eig || !state->u ||
      !state->strain || !state->stress || !state->H || !state->damage)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (prm->eig_mode == FFTMECH_EIG_PRESCRIBED && !prm->eig_field)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "eig_field is required for PRESCRIBED");
  for (int i = 0; i < 3; ++i) fill_info_defaults(&info[i]);
  const size_t N = (size_t)ctx->N, es = esize(ctx), nv = nvoigt(ctx);
  cudaStream_t st = ctx->stream;
  // stage everything once for the whole step
  void *dphase, *dc, *dcppt, *deig, *du, *dstrain, *dstress, *dH, *dd, *dmask = nullptr, *deigf = nullptr;
  if ((rc = stage_in(ctx, ST_PHASE, state->phase, N, true, &dphase)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_C, state->c, N * 8, true, &dc)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_CPPT, state->c_ppt, N * es, true, &dcppt)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_EIG, state->eig, N * es, true, &deig)) != FFTMECH_OK) return rc;
  if ((rc = stage_in(ctx, ST_U, state->u, 2 * N * 8, true, &du)) != FFTMECH_OK) return rc;
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
                                 (double*)dc, &info[0])
        : diffusion_impl<float>(ctx, (const uint8_t*)dphase, prm->diffusion_mode, prm->grad_c_mac,
                                prm->c_macro, prm->dt, (const uint8_t*)dmask, prm->dirichlet_value,
                                (double*)dc, &info[0]);
    if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
    track(s);
  }
  // 2. precipitation and eigenstrain
  if (prm->eig_mode == FFTMECH_EIG_FROM_PRECIPITATE) {
    ProfScope _ps(ctx, FFTMECH_K_OTHER);
    if (fp64)
      CK(launch_precipitate<double>(ctx->N, (const uint8_t*)dphase, (const double*)dc, ctx->mat.S_sol,
                                    ctx->mat.M_ppt, (double*)dcppt, (double*)deig, st));
    else
      CK(launch_precipitate<float>(ctx->N, (const uint8_t*)dphase, (const double*)dc, ctx->mat.S_sol,
                                   ctx->mat.M_ppt, (float*)dcppt, (float*)deig, st));
  } else {
    ProfScope _ps(ctx, FFTMECH_K_OTHER);
    if (fp64)
      CK(launch_scale_copy<double>(ctx->N, (const double*)deigf, prm->eig_scale, (double*)deig, st));
    else
      CK(launch_scale_copy<float>(ctx->N, (const float*)deigf, prm->eig_scale, (float*)deig, st));
  }
  // 3. equilibrium with the stiffness degraded by the current damage
  {
    fftmech_status s = fp64
        ? equilibrium_impl<double>(ctx, (const uint8_t*)dphase, (const double*)deig, (const double*)dd,
                                   prm->eps_mac, (double*)du, (double*)dstrain, (double*)dstress, &info[1])
        : equilibrium_impl<float>(ctx, (const uint8_t*)dphase, (const float*)deig, (const double*)dd,
                                  prm->eps_mac, (double*)du, (float*)dstrain, (float*)dstress, &info[1]);
    if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
    track(s);
  }
  // 4. history and phase field
  {
    fftmech_status s = fp64
        ? phasefield_impl<double>(ctx, (const double*)dstrain, (const double*)deig, (const uint8_t*)dphase,
                                  (double*)dH, (double*)dd, &info[2])
        : phasefield_impl<float>(ctx, (const float*)dstrain, (const float*)deig, (const uint8_t*)dphase,
                                 (float*)dH, (double*)dd, &info[2]);
    if (s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG) return s;
    track(s);
  }
  if ((rc = stage_out(ctx, state->c, dc, N * 8)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->c_ppt, dcppt, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->eig, deig, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->u, du, 2 * N * 8)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->strain, dstrain, nv * N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->stress, dstress, nv * N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->H, dH, N * es)) != FFTMECH_OK) return rc;
  if ((rc = stage_out(ctx, state->damage, dd, N * 8)) != FFTMECH_OK) return rc;
  CK(cudaStreamSynchronize(st));
  return worst;
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
      Spec2<double> sp{};
      e = launch_rowfft_f<double>(px.fam, nx, ny, (cx<double>*)data, dev_plan<double>(px), inverse, sh, st);
      if (e == cudaSuccess && ny > 1)
        e = launch_colpass_f<double>(py.fam, nx, ny, (cx<double>*)data, dev_plan<double>(py), sp, sh, COL_PLAIN,
                                   inverse, nullptr, nullptr, st);
    } else {
      Spec2<float> sp{};
      e = launch_rowfft_f<float>(px.fam, nx, ny, (cx<float>*)data, dev_plan<float>(px), inverse, sh, st);
      if (e == cudaSuccess && ny > 1)
        e = launch_colpass_f<float>(py.fam, nx, ny, (cx<float>*)data, dev_plan<float>(py), sp, sh, COL_PLAIN,
                                  inverse, nullptr, nullptr, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = FFTMECH_ERR_CUDA;
  }
  free_plan(px);
  free_plan(py);
  return rc;
}

}  // extern "C"
