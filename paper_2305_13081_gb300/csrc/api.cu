// C ABI of libfftmech: contexts, FFT plans, workspace, the device-driven PCG
// (run as one CUDA graph with conditional nodes, or host-driven with the
// same kernels) and the entry points declared in include/fftmech.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
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

// Plans of the stand-alone transform, kept per (device, length) for the life
// of the process (the device twiddles of a length are made on its first use).
std::mutex g_plan_mu;
std::map<std::pair<int, int>, HostPlan> g_plans;

cudaError_t cached_plan(int dev, int n, HostPlan& out) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find({dev, n});
  if (it == g_plans.end()) {
    HostPlan p;
    const cudaError_t e = make_plan(n, p);
    if (e != cudaSuccess) {
      free_plan(p);
      return e;
    }
    it = g_plans.emplace(std::make_pair(dev, n), p).first;
  }
  out = it->second;
  return cudaSuccess;
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

// The three solves of a staggered step; each keeps its own record (solver
// scalars, post-processing sums, device timestamps) so that one read after
// the whole step reports all three.
enum SolveKind { SK_DIFF = 0, SK_EQ = 1, SK_PF = 2, SK_COUNT = 3 };
// Operations with a cached graph.
enum OpKind { OP_STEP = 0, OP_DIFF = 1, OP_EQ = 2, OP_PF = 3, OP_BAR = 4, OP_COUNT = 5 };

constexpr int kResultsPerProblem = 16;

// Kernel launches of a captured operation: those outside any conditional
// node, and per solve the launches directly inside each conditional body
// (one execution of that body). A replay's total follows from the solves'
// records (iterations, replacements, restarts).
struct LaunchCount {
  long long fixed = 0;
  long long body[SK_COUNT][LF_COUNT] = {};
};

struct GraphCache {
  std::vector<unsigned char> key;  // the arguments the graph was captured with
  cudaGraphExec_t exec = nullptr;
  LaunchCount lc;
};

// What the host needs to turn the records of the last operation into
// fftmech_solve_info (kept when the operation is enqueued).
struct LastOp {
  int valid = 0;
  int ran[SK_COUNT] = {0, 0, 0};
  int diff_mode = 0;
  double c_macro = 0.0;
  const LaunchCount* lc = nullptr;  // the operation ran as this cached graph
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
  void* p = nullptr;     // search direction (updated in place by the direction kernel)
  void* pn = nullptr;    // 2D: the new direction of the fused direction-stencil kernel
  // fused direction-stencil kernel: -1 as launch_mode bit 1 asks, 0 split,
  // 1 fused (fftmech_autotune's choice); ds_rule: its rows per block by the
  // host's rule (0: no fused kernel on this grid)
  int ds_choice = -1;
  int ds_rule = 0;
  void* S = nullptr;
  void* q = nullptr;     // K p of the split iteration
  void* g = nullptr;
  float* uh = nullptr;   // MIXED iterate, high part
  float* ul = nullptr;   // MIXED iterate, low part
  double* phi = nullptr;
  double* Hd = nullptr;
  double* cn = nullptr;
  void* az = nullptr;     // 3D: D h along z (reference-medium preconditioner)
  void* lamx = nullptr;
  void* lamy = nullptr;
  void* lamz = nullptr;     // 3D: lambda_z(kz)
  void* lamc3 = nullptr;    // 3D: lambda_x per spectral column, D = 3 / D = 1 rows
  void* lamc1 = nullptr;
  void* wcol3 = nullptr;    // 3D: Parseval weight per spectral column
  void* wcol1 = nullptr;
  void* ax = nullptr;       // 2D: D h per column kx = 0 .. nx / 2 (complex), reference medium
  void* ay = nullptr;       // 2D: D h per row ky (complex)
  double rho = 0;           // lambda / mu of the solid (reference medium)
  int ms_cw = 0, ms_threads = 0;  // reference-medium column pass: strip width, threads (0: unavailable)
  int ms3_cw = 0, ms3_threads = 0;  // reference-medium z pass (3D): strip width, threads (0: unavailable)
  double* partials = nullptr;
  double* partials_col = nullptr;  // 2D column pass (deferred reductions)
  double* m0b = nullptr;       // per-problem preconditioner constants
  double* m1b = nullptr;
  int* mode = nullptr;         // per-problem iteration modes (0, 1 reliable update, 2 restart)
  SolverScalars* sc = nullptr;
  int* flags = nullptr;        // loop flags (LF_COUNT ints)
  int* h_flags = nullptr;      // pinned copy read by the host-driven loop
  // record block: SolverScalars[SK_COUNT][B], double[SK_COUNT][16 B],
  // unsigned long long[SK_COUNT][2]; copied to the pinned h_rec at the end
  // of every operation
  unsigned char* rec = nullptr;
  unsigned char* h_rec = nullptr;
  size_t rec_bytes = 0;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};  // streams that capture conditional bodies
  GraphCache gc[OP_COUNT];
  bool graph_off = false;   // a graph failed to build or launch: host-driven from then on
  long long graph_builds = 0, graph_launches = 0;
  long long graph_kernels = 0;  // kernels run by graph replays whose reports were read
  const LaunchCount* pending_lc = nullptr;  // set by run_op for the operation just enqueued
  char graph_err[256] = {0};
  LastOp last;
  char tune_desc[160] = {0};  // the launch shapes in use (after fftmech_autotune or a cached choice)
  Staging stage[ST_COUNT];
  // instrumentation
  bool prof = false;
  long long launches[FFTMECH_K_COUNT] = {0};
  double prof_ms[FFTMECH_K_COUNT] = {0};
  struct Pending { int k; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  char err[512] = {0};
};

// Staggered steps of several contexts as one graph (parallel branches).
struct fftmech_group {
  std::vector<fftmech_ctx*> ctxs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  std::vector<LaunchCount> lc;
  long long builds = 0, launches = 0, kernels = 0;
  char err[512] = {0};
};

// The device arrays and constants of a macroscale bar (Sec. 3.2).
struct BarDev {
  int M = 0;
  double dX = 0, dt = 0, flux_in = 0;
  double* c = nullptr;     // M + 1 nodal concentrations
  double* cbar = nullptr;  // M element concentrations
  double* G = nullptr;     // 3 M element gradients
};

struct fftmech_bar {
  fftmech_ctx* ctx = nullptr;
  BarDev d;
  double* mem = nullptr;
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

#define RC(...)                              \
  do {                                        \
    const fftmech_status _r = (__VA_ARGS__);  \
    if (_r != FFTMECH_OK) return _r;          \
  } while (0)

size_t esize(const fftmech_ctx* ctx) { return ctx->prec == FFTMECH_FP64 ? 8 : 4; }
int nvoigt(const fftmech_ctx* ctx) { return ctx->dim == 2 ? 3 : 6; }

// record block layout
size_t rec_sc_off(const fftmech_ctx* c, int k) { return (size_t)k * c->B * sizeof(SolverScalars); }
size_t rec_res_off(const fftmech_ctx* c, int k) {
  return (size_t)SK_COUNT * c->B * sizeof(SolverScalars) + (size_t)k * kResultsPerProblem * c->B * sizeof(double);
}
size_t rec_stamp_off(const fftmech_ctx* c, int k) {
  return (size_t)SK_COUNT * c->B * sizeof(SolverScalars) + (size_t)SK_COUNT * kResultsPerProblem * c->B * sizeof(double) +
         (size_t)k * 2 * sizeof(unsigned long long);
}
size_t rec_total(const fftmech_ctx* c) { return rec_stamp_off(c, SK_COUNT); }
double* res_dev(fftmech_ctx* c, int k) { return reinterpret_cast<double*>(c->rec + rec_res_off(c, k)); }
unsigned long long* stamp_dev(fftmech_ctx* c, int k) {
  return reinterpret_cast<unsigned long long*>(c->rec + rec_stamp_off(c, k));
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller buffer: the pointer itself if it is device memory,
// else a staging buffer (allocated on first use, copied in when `in`).
// Output copy-back is done by `stage_out`.
fftmech_status stage_in(fftmech_ctx* ctx, StageSlot slot, const void* ptr, size_t bytes, bool in,
                        void** dev) {
  if (!ptr) { *dev = nullptr; return FFTMECH_OK; }
  if (is_device_ptr(ptr)) { *dev = const_cast<void*>(ptr); return FFTMECH_OK; }
  Staging& s = ctx->stage[slot];
  if (s.bytes < bytes) {
    if (s.dev) {
      CK(cudaStreamSynchronize(ctx->stream));
      CK(cudaFree(s.dev));
    }
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

// Counts one launch of class k and, when profiling, brackets it with events
// (host-driven execution only: profiling turns the graph path off).
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
  {
    // D h = e^{i theta} - 1 per mode (reference-medium preconditioner):
    // columns 0 .. nx / 2 along x, every frequency along y and z
    auto dh = [](int k, int n, T* out) {
      const double th = 2.0 * M_PI * k / n;
      out[0] = (T)(std::cos(th) - 1.0);
      out[1] = (T)std::sin(th);
    };
    const int H = ctx->nx / 2 + 1;
    std::vector<T> ax(2 * H), ay(2 * ctx->ny), az(2 * ctx->nz);
    for (int k = 0; k < H; ++k) dh(k, ctx->nx, &ax[2 * k]);
    for (int k = 0; k < ctx->ny; ++k) dh(k, ctx->ny, &ay[2 * k]);
    for (int k = 0; k < ctx->nz; ++k) dh(k, ctx->nz, &az[2 * k]);
    CK(cudaMemcpy(ctx->ax, ax.data(), sizeof(T) * ax.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->ay, ay.data(), sizeof(T) * ay.size(), cudaMemcpyHostToDevice));
    if (ctx->dim == 3) CK(cudaMemcpy(ctx->az, az.data(), sizeof(T) * az.size(), cudaMemcpyHostToDevice));
  }
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


// ---------------------------------------------------------------- emission
// Where the launches of an operation go. graph: the stream is capturing into
// `g` (the context's stream for the top level, a side stream for the body of
// a conditional node); the loops become conditional nodes whose conditions
// the kernels set. Otherwise the host drives the same loops and reads the
// kernels' loop flags from device memory.
struct Emit {
  fftmech_ctx* ctx;
  cudaStream_t st;
  bool graph;
  cudaGraph_t g;
  int depth;
  LoopCtl ctl;
  LaunchCount* lc;  // graph mode: launches counted per level
  int sk;           // solve being emitted
  int level;        // -1 outside conditional nodes, else the flag of the innermost one
};

inline void em_count(Emit& em) {
  if (!em.graph || !em.lc) return;
  if (em.level < 0) em.lc->fixed += 1;
  else em.lc->body[em.sk][em.level] += 1;
}

#define EM_LAUNCH(EM, KC, CALL)        \
  do {                                 \
    if (!(EM).graph) {                 \
      ProfScope _ps(ctx, KC);          \
      CK(CALL);                        \
    } else {                           \
      CK(CALL);                        \
      em_count(EM);                    \
    }                                  \
  } while (0)

Emit eager_emit(fftmech_ctx* ctx) {
  Emit e{};
  e.ctx = ctx;
  e.st = ctx->stream;
  e.graph = false;
  e.ctl.flags = ctx->flags;
  e.ctl.direct = ctx->B == 1;
  e.lc = nullptr;
  e.sk = 0;
  e.level = -1;
  return e;
}

// Conditional handle for flag k in the graph being captured (graph mode);
// `reset`: the condition returns to `value` at every launch of the graph.
fftmech_status em_handle(Emit& em, int k, bool reset = false, unsigned int value = 0) {
  if (!em.graph) return FFTMECH_OK;
  fftmech_ctx* ctx = em.ctx;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, em.g, value, reset ? cudaGraphCondAssignDefault : 0));
  em.ctl.h[k] = (unsigned long long)h;
  em.ctl.have |= 1u << k;
  return FFTMECH_OK;
}

// Graph mode: a conditional node (WHILE or IF on flag k) after everything
// captured so far, its body captured by `body` on a side stream.
template <typename F>
fftmech_status em_cond(Emit& em, int k, cudaGraphConditionalNodeType type, F&& body) {
  fftmech_ctx* ctx = em.ctx;
  if (em.depth >= 3) return set_err(ctx, FFTMECH_ERR_CUDA, "conditional nodes nested too deeply");
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(em.st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return set_err(ctx, FFTMECH_ERR_CUDA, "stream is not capturing");
  // the parameter struct holds a union without a default constructor:
  // zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = (cudaGraphConditionalHandle)em.ctl.h[k];
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  cudaGraph_t body_g = p.conditional.phGraph_out[0];
  cudaStream_t side = ctx->side[em.depth];
  CK(cudaStreamBeginCaptureToGraph(side, body_g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  Emit sub = em;
  sub.st = side;
  sub.g = body_g;
  sub.depth = em.depth + 1;
  sub.level = k;
  const fftmech_status rc = body(sub);
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(side, &out);
  if (rc != FFTMECH_OK) return rc;
  CK(e);
  CK(cudaStreamUpdateCaptureDependencies(em.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return FFTMECH_OK;
}

// Host-driven execution: the kernels' loop flags (synchronises the stream).
fftmech_status poll_flags(Emit& em, int* out) {
  fftmech_ctx* ctx = em.ctx;
  CK(cudaMemcpyAsync(ctx->h_flags, ctx->flags, sizeof(int) * LF_COUNT, cudaMemcpyDeviceToHost, em.st));
  CK(cudaStreamSynchronize(em.st));
  prof_flush(ctx);
  for (int k = 0; k < LF_COUNT; ++k) out[k] = ctx->h_flags[k];
  return FFTMECH_OK;
}

// Whether a 2D solve may run the fused direction-stencil kernel (the grid
// has one, and launch_mode bit 1 or fftmech_autotune chose it).
inline bool ds_active(const fftmech_ctx* ctx) {
  if (ctx->lshape.L_ds <= 0) return false;
  return ctx->ds_choice < 0 ? (ctx->opts.launch_mode & 2) != 0 : ctx->ds_choice == 1;
}

// ---------------------------------------------------------------- PCG
// Preconditioned CG on the potential for every problem of the batch.
// Launch sequence (graph form; the host-driven form runs the same launches
// and reads the flags after every iteration):
//   scalars, [MIXED: iterate split], <f, M^-1 f>, first residual, zero-RHS
//   case, first direction (p = z)               -> LF_LOOP, LF_REPLACE, LF_GATE
//   WHILE LF_OUTER:
//     conditions from memory
//     WHILE LF_LOOP (ordinary iterations):
//       stencil (q = K p, <p, K p>), update (u += alpha p, r -= alpha q,
//       x-FFT), column pass (multiplier, <r, M^-1 r>), direction
//     IF LF_REPLACE (reliable update): stencil, update of the iterate only,
//       true residual, column pass, direction
//     IF LF_GATE: true residual of the problems that stopped unchecked
//     restart gate
//     IF LF_RESTART: restart from the true residual, first direction
//   [MIXED: iterate merge]
// An ordinary iteration has no conditional node inside it, so its kernels
// stay chained by programmatic dependent launches. Where the 2D iteration
// is latency-bound the direction and the next iteration's stencil are one
// kernel: an iteration is then update, column pass, direction-stencil.
// The true residual is FP64 on the FP64 path and double-float on the mixed
// one.
// Every decision (convergence, iteration limit, reliable update, restart) is
// taken on the device; a problem that has stopped makes every kernel return
// at once while the others continue.
template <typename T, int D>
fftmech_status emit_pcg(Emit& em, const Op<T>& op_in, double* u, const Spec<T>& sp_in) {
  fftmech_ctx* ctx = em.ctx;
  const DepLaunchScope dep((ctx->opts.launch_mode & 1) == 0);
  const int B = ctx->B;
  FftPlanDev<T> px = dev_plan<T>(ctx->px), py = dev_plan<T>(ctx->py), pz = dev_plan<T>(ctx->pz);
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
  const bool three = ctx->dim == 3;
  if (three) {
    sp.lamc = (const T*)(D == 1 ? ctx->lamc1 : ctx->lamc3);
    sp.wcol = (const T*)(D == 1 ? ctx->wcol1 : ctx->wcol3);
    sp.lamj = (const T*)ctx->lamy;
    sp.laml = (const T*)ctx->lamz;
  }
  Vec2<T> v{};
  v.u = u;
  v.uh = ctx->uh;
  v.ul = ctx->ul;
  v.r = (T*)ctx->r;
  v.p_in = (const T*)ctx->p;
  v.p_out = (T*)ctx->p;
  v.S = (cx<T>*)ctx->S;
  v.q = (T*)ctx->q;
  v.partials = ctx->partials;
  v.sc = ctx->sc;
  v.mode = ctx->mode;
  v.pcol = ctx->partials_col;
  // Deferred reductions where the grid is latency-bound (up to 2^21 voxels
  // per launch): the stencil's <p, K p> summed by the update kernel (2D and
  // 3D), the column pass's <r, M^-1 r> by the next direction kernel (2D).
  // Larger grids keep the last-block reductions: there every consumer block
  // re-reading all partials costs more than the ticket saves.
  const bool small = (long long)ctx->N * B <= (1LL << 21);
  const bool defer = small && !three;
  // there the direction and the stencil can run as one kernel
  // (launch_mode bit 1, or fftmech_autotune's choice): it writes the new
  // direction to pn, and the update kernel, which reads it, copies it back
  // to p for the next direction
  const bool fused = defer && ds_active(ctx);
  // reference-medium preconditioner: elasticity (2D column pass, 3D z pass)
  const bool ms = D == 2 && !three && ctx->opts.precond == FFTMECH_PRECOND_REFERENCE && ctx->ms_cw > 0;
  const bool ms3 = D == 3 && three && ctx->opts.precond == FFTMECH_PRECOND_REFERENCE && ctx->ms3_cw > 0;
  if (ms || ms3) {
    sp.ax = (const cx<T>*)ctx->ax;
    sp.ay = (const cx<T>*)ctx->ay;
    sp.az = (const cx<T>*)ctx->az;
    sp.rho_t = (T)ctx->rho;
  }
  const int ncol_blocks = !defer ? 0
                          : ms   ? colpass_ms_blocks(ctx->nx, ctx->ms_cw)
                                 : (ctx->nx + ctx->shape.cols - 1) / ctx->shape.cols;
  v.nsten = !small ? 0
            : three ? sten3_blocks(ctx->nx, ctx->ny, ctx->nz, ctx->sshape)
            : fused ? (ctx->ny + ctx->lshape.L_ds - 1) / ctx->lshape.L_ds
                    : sten2_blocks(ctx->nx, ctx->ny, ctx->sshape);
  const long long nU = (long long)D * ctx->N * B;
  const bool mixed = sizeof(T) == 4;
  const bool reliable = mixed && ctx->opts.replace_residual != 0;
  const int fx = ctx->px.fam, fy = ctx->py.fam, fz = ctx->pz.fam;
  const Shape2& sh = ctx->shape;
  const Shape3& sh3 = ctx->shape3;
  const LineShape& lsh = ctx->lshape;
  const StenShape& ssh = ctx->sshape;
  auto residual = [&](int zero_u, int filter, cudaStream_t st) -> cudaError_t {
    if constexpr (D == 3) return launch3_residual_f<T, 3>(fx, op, v, px, sh3, zero_u, filter, st);
    else if constexpr (D == 2) return launch_residual_f<T, 2>(fx, op, v, px, sh, zero_u, filter, st);
    else
      return three ? launch3_residual_f<T, 1>(fx, op, v, px, sh3, zero_u, filter, st)
                   : launch_residual_f<T, 1>(fx, op, v, px, sh, zero_u, filter, st);
  };
  auto direction = [&](const Vec2<T>& va, cudaStream_t st) -> cudaError_t {
    if (fused) {
      Vec2<T> vf = va;
      vf.p_out = (T*)ctx->pn;
      if constexpr (D == 2) return launch_xds_f<T, 2>(fx, op, vf, px, lsh, st);
      else if constexpr (D == 1) return launch_xds_f<T, 1>(fx, op, vf, px, lsh, st);
    }
    if constexpr (D == 3) return launch_xdir_f<T, 3, 3>(fx, op, va, px, lsh, st);
    else if constexpr (D == 2) return launch_xdir_f<T, 2, 2>(fx, op, va, px, lsh, st);
    else
      return three ? launch_xdir_f<T, 1, 3>(fx, op, va, px, lsh, st) : launch_xdir_f<T, 1, 2>(fx, op, va, px, lsh, st);
  };
  auto stencil = [&](const Vec2<T>& vs, cudaStream_t st) -> cudaError_t {
    if constexpr (D == 3) return launch_sten3<T, 3>(op, vs, ssh, st);
    else if constexpr (D == 2) return launch_sten2<T, 2>(op, vs, ssh, st);
    else return three ? launch_sten3<T, 1>(op, vs, ssh, st) : launch_sten2<T, 1>(op, vs, ssh, st);
  };
  auto update = [&](const Vec2<T>& vu_in, cudaStream_t st) -> cudaError_t {
    Vec2<T> vu = vu_in;
    if (fused) {
      vu.p_in = (const T*)ctx->pn;
      vu.p_copy = (T*)ctx->p;
    }
    if constexpr (D == 3) return launch_xupd_f<T, 3, 3>(fx, op, vu, px, lsh, st);
    else if constexpr (D == 2) return launch_xupd_f<T, 2, 2>(fx, op, vu, px, lsh, st);
    else
      return three ? launch_xupd_f<T, 1, 3>(fx, op, vu, px, lsh, st) : launch_xupd_f<T, 1, 2>(fx, op, vu, px, lsh, st);
  };
  // 2D: one column pass; 3D: y-FFT, z pass (multiplier, <r, M^-1 r>), y-IFFT
  auto colpass = [&](int mode, cudaStream_t st) -> cudaError_t {
    if (ms)
      return launch_colpass_ms_f<T>(fy, ctx->nx, ctx->ny, v.S, py, sp, ctx->ms_cw, ctx->ms_threads, B, mode,
                                    ctx->partials_col, ctx->sc, ctx->mode, st);
    if (!three)
      return launch_colpass_f<T>(fy, ctx->nx, ctx->ny, v.S, py, sp, sh, mode, 0, ctx->partials_col, ctx->sc, ctx->mode,
                                 st);
    cudaError_t e = launch3_lines_f<T>(fy, v.S, sh3, D, 1, 0, py, sp, mode, nullptr, ctx->sc, ctx->mode, st);
    if (e != cudaSuccess) return e;
    e = ms3 ? launch3_zpass_ms_f<T>(fz, v.S, sh3.sst, ctx->nx, ctx->ny, ctx->nz, (int)nxs_of(ctx->nx, 3), pz, sp,
                                    ctx->ms3_cw, ctx->ms3_threads, B, mode, ctx->partials, ctx->sc, ctx->mode, st)
            : launch3_lines_f<T>(fz, v.S, sh3, D, 2, 1, pz, sp, mode, ctx->partials, ctx->sc, ctx->mode, st);
    if (e != cudaSuccess || mode == COL_NORM || mode == COL_TRUENORM) return e;
    return launch3_lines_f<T>(fy, v.S, sh3, D, 1, 2, py, sp, mode, nullptr, ctx->sc, ctx->mode, st);
  };

  // set-up: scalars, first residual
  const double tol = ctx->opts.tol;
  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_sc_init(ctx->sc, B, tol * tol, ctx->opts.max_iter, reliable ? 1 : 0, em.st));
  if (mixed) EM_LAUNCH(em, FFTMECH_K_OTHER, launch_df_split(nU, u, ctx->uh, ctx->ul, em.st));
  EM_LAUNCH(em, FFTMECH_K_RESIDUAL, residual(1, 0, em.st));
  EM_LAUNCH(em, FFTMECH_K_COLUMN, colpass(COL_NORM, em.st));
  EM_LAUNCH(em, FFTMECH_K_RESIDUAL, residual(0, 0, em.st));
  EM_LAUNCH(em, FFTMECH_K_COLUMN, colpass(COL_INIT, em.st));
  EM_LAUNCH(em, FFTMECH_K_OTHER,
            launch_zero_rhs(u, mixed ? ctx->uh : nullptr, mixed ? ctx->ul : nullptr, (long long)D * ctx->N, ctx->sc, B,
                            op.mask ? 1 : 0, em.st));

  // first direction after the first residual or a restart (beta = 0)
  auto first_direction = [&](Emit& e) -> fftmech_status {
    Vec2<T> va = v;
    va.ncol = 0;
    va.ctl = e.ctl;
    EM_LAUNCH(e, FFTMECH_K_DIRECTION, direction(va, e.st));
    if (B > 1) EM_LAUNCH(e, FFTMECH_K_OTHER, launch_loopctl(ctx->sc, ctx->mode, B, va.ctl, e.st));
    return FFTMECH_OK;
  };
  // One iteration, ending with the next direction. In a replacement
  // iteration (not plain) the update kernel moves only the iterate of the
  // problems in mode 1 and the FP64 true residual becomes their residual.
  // Ordinary iterations run only while no problem has a replacement due.
  auto iteration = [&](Emit& e, bool plain) -> fftmech_status {
    Vec2<T> vi = v;
    vi.ctl = e.ctl;
    if (!fused) EM_LAUNCH(e, FFTMECH_K_STENCIL, stencil(vi, e.st));
    EM_LAUNCH(e, FFTMECH_K_UPDATE, update(vi, e.st));
    if (!plain) EM_LAUNCH(e, FFTMECH_K_RESIDUAL, residual(0, 1, e.st));
    EM_LAUNCH(e, FFTMECH_K_COLUMN, colpass(defer ? (COL_ITER | COL_DEFER) : COL_ITER, e.st));
    vi.ncol = ncol_blocks;
    EM_LAUNCH(e, FFTMECH_K_DIRECTION, direction(vi, e.st));
    if (B > 1) EM_LAUNCH(e, FFTMECH_K_OTHER, launch_loopctl(ctx->sc, ctx->mode, B, vi.ctl, e.st));
    return FFTMECH_OK;
  };
  // End of an outer round: the FP64 true residual of every problem that has
  // stopped since the last check (only when the last decision saw one: in
  // a batch most rounds end with a replacement and check nothing), then the
  // restart gate (a no-op while some problem is active)
  const int max_rounds = ctx->opts.max_iter + 64;
  auto truecheck = [&](Emit& e) -> fftmech_status {
    EM_LAUNCH(e, FFTMECH_K_RESIDUAL, residual(0, 2, e.st));
    EM_LAUNCH(e, FFTMECH_K_COLUMN, colpass(COL_TRUENORM, e.st));
    return FFTMECH_OK;
  };
  auto gate = [&](Emit& e) -> fftmech_status {
    EM_LAUNCH(e, FFTMECH_K_OTHER, launch_gate(ctx->sc, ctx->mode, B, e.ctl, max_rounds, e.st));
    return FFTMECH_OK;
  };
  auto restart = [&](Emit& e) -> fftmech_status {
    EM_LAUNCH(e, FFTMECH_K_RESIDUAL, residual(0, 1, e.st));
    EM_LAUNCH(e, FFTMECH_K_COLUMN, colpass(COL_RESTART, e.st));
    EM_LAUNCH(e, FFTMECH_K_OTHER, launch_clear_modes(ctx->mode, B, e.st));
    return first_direction(e);
  };

  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_set_flag(em.ctl, LF_OUTER, 1, em.st));
  RC(first_direction(em));
  if (em.graph) {
    // WHILE outer {
    //   conditions from memory; WHILE loop { ordinary iteration }
    //   IF replace { replacement iteration }
    //   IF gate { true residuals }; gate; IF restart { restart, first direction } }
    // Every condition is set by kernels of its own graph or of a body one
    // level down.
    Emit top = em;
    RC(em_handle(top, LF_OUTER));
    EM_LAUNCH(top, FFTMECH_K_OTHER, launch_set_flag(top.ctl, LF_OUTER, 1, top.st));
    RC(em_cond(top, LF_OUTER, cudaGraphCondTypeWhile, [&](Emit& o) -> fftmech_status {
      RC(em_handle(o, LF_LOOP));
      RC(em_handle(o, LF_REPLACE));
      RC(em_handle(o, LF_RESTART));
      RC(em_handle(o, LF_GATE));
      EM_LAUNCH(o, FFTMECH_K_OTHER, launch_sync_flags(o.ctl, o.st));
      RC(em_cond(o, LF_LOOP, cudaGraphCondTypeWhile, [&](Emit& l) { return iteration(l, true); }));
      RC(em_cond(o, LF_REPLACE, cudaGraphCondTypeIf, [&](Emit& r) { return iteration(r, false); }));
      RC(em_cond(o, LF_GATE, cudaGraphCondTypeIf, truecheck));
      RC(gate(o));
      return em_cond(o, LF_RESTART, cudaGraphCondTypeIf, restart);
    }));
  } else {
    // the same launches; the host reads the kernels' decisions after every
    // iteration (an ordinary iteration must not start once a replacement is
    // due)
    const long long cap = (long long)ctx->opts.max_iter + 8;  // guard of the host loop
    int f[LF_COUNT];
    long long total = 0;
    for (;;) {
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch_sync_flags(em.ctl, em.st));
      RC(poll_flags(em, f));
      while (f[LF_LOOP]) {
        RC(iteration(em, true));
        if (++total > cap) return set_err(ctx, FFTMECH_ERR_CUDA, "PCG loop did not stop within its iteration limit");
        RC(poll_flags(em, f));
      }
      if (f[LF_REPLACE]) {
        RC(iteration(em, false));
        if (++total > cap) return set_err(ctx, FFTMECH_ERR_CUDA, "PCG loop did not stop within its iteration limit");
        RC(poll_flags(em, f));
      }
      if (f[LF_GATE]) RC(truecheck(em));
      RC(gate(em));
      RC(poll_flags(em, f));
      if (!f[LF_OUTER]) break;
      if (f[LF_RESTART]) RC(restart(em));
    }
  }
  if (mixed) EM_LAUNCH(em, FFTMECH_K_OTHER, launch_df_merge(nU, ctx->uh, ctx->ul, u, em.st));
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

// Start of a solve's record: device clock.
fftmech_status rec_begin(Emit& em, int kind) {
  fftmech_ctx* ctx = em.ctx;
  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_stamp(stamp_dev(ctx, kind), em.st));
  return FFTMECH_OK;
}
// End of a solve's record: its solver scalars and the device clock.
fftmech_status rec_end(Emit& em, int kind) {
  fftmech_ctx* ctx = em.ctx;
  CK(cudaMemcpyAsync(ctx->rec + rec_sc_off(ctx, kind), ctx->sc, sizeof(SolverScalars) * ctx->B,
                     cudaMemcpyDeviceToDevice, em.st));
  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_stamp(stamp_dev(ctx, kind) + 1, em.st));
  return FFTMECH_OK;
}
// End of an operation: the record block to the pinned host copy.
fftmech_status rec_publish(Emit& em) {
  fftmech_ctx* ctx = em.ctx;
  CK(cudaMemcpyAsync(ctx->h_rec, ctx->rec, ctx->rec_bytes, cudaMemcpyDeviceToHost, em.st));
  return FFTMECH_OK;
}

// ---------------------------------------------------------------- solves (enqueue)
template <typename T>
fftmech_status enqueue_equilibrium(Emit& em, const uint8_t* phase, const T* eig, const double* damage,
                                   const double* eps_mac, double* u, T* strain, T* stress) {
  fftmech_ctx* ctx = em.ctx;
  em.sk = SK_EQ;
  RC(rec_begin(em, SK_EQ));
  const int B = ctx->B;
  const long long NB = ctx->N * B;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  op.eig = eig;
  for (int k = 0; k < nvoigt(ctx); ++k) op.E[k] = eps_mac[k];
  if (damage) {
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch_degradation<T>(NB, damage, ctx->mat.kappa, (T*)ctx->g, em.st));
    op.g = (const T*)ctx->g;
  }
  Spec<T> sp{};
  sp.m0 = 0.0;
  sp.m1 = 1.0 / (ctx->h * ctx->h);
  const bool three = ctx->dim == 3;
  RC(three ? emit_pcg<T, 3>(em, op, u, sp) : emit_pcg<T, 2>(em, op, u, sp));
  double* res = res_dev(ctx, SK_EQ);
  if (three)
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch3_el_output<T>(op, B, u, strain, stress, ctx->partials, res, ctx->sc, em.st));
  else
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch_el_output<T>(op, B, u, strain, stress, ctx->partials, res, ctx->sc, em.st));
  return rec_end(em, SK_EQ);
}

template <typename T>
fftmech_status enqueue_diffusion(Emit& em, const uint8_t* phase, int mode, const double* grad_c_mac, double c_macro,
                                 double dt, const uint8_t* mask, double cD, double* c, const double* Gp = nullptr,
                                 const double* cmp = nullptr) {
  fftmech_ctx* ctx = em.ctx;
  em.sk = SK_DIFF;
  if (mode == FFTMECH_DIFF_TRANSIENT && !(dt > 0))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt must be > 0 for TRANSIENT");
  RC(rec_begin(em, SK_DIFF));
  const int B = ctx->B;
  const long long NB = ctx->N * B;
  const bool three = ctx->dim == 3;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  op.h = ctx->h_diff;
  op.kap[0] = ctx->mat.D_pore;
  op.kap[1] = ctx->mat.D_solid;
  const double ih2 = 1.0 / (ctx->h_diff * ctx->h_diff);
  double* res = res_dev(ctx, SK_DIFF);
  Spec<T> sp{};
  if (mode == FFTMECH_DIFF_HOMOGENISE) {
    op.G[0] = grad_c_mac[0];
    op.G[1] = grad_c_mac[1];
    op.G[2] = three ? grad_c_mac[2] : 0.0;
    op.Gp = Gp;
    op.cmp = cmp;
    sp.m0 = 0.0;
    sp.m1 = ih2;
    RC(emit_pcg<T, 1>(em, op, ctx->phi, sp));
    if (three) {
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch3_diff_stats<T>(op, B, ctx->phi, ctx->h_diff, c_macro, ctx->partials, res,
                                                           ctx->sc, em.st));
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch3_diff_write_c(ctx->nx, ctx->ny, ctx->nz, B, phase, ctx->phi, ctx->h_diff,
                                                          op.G, Gp, res, c, em.st));
    } else {
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch_diff_stats<T>(op, B, ctx->phi, ctx->h_diff, c_macro, ctx->partials, res,
                                                          ctx->sc, em.st));
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch_diff_write_c(ctx->nx, ctx->ny, B, phase, ctx->phi, ctx->h_diff, op.G[0],
                                                         op.G[1], Gp, res, c, em.st));
    }
    return rec_end(em, SK_DIFF);
  }
  // TRANSIENT (backward Euler, not in the paper): per-problem porosity ->
  // mean diffusivity of the preconditioner (on device)
  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_pf_stats(ctx->N, B, phase, nullptr, ctx->partials, res, ctx->sc,
                                                 ctx->mat.D_pore, ctx->mat.D_solid, ih2, ctx->m1b, em.st));
  if (mask) EM_LAUNCH(em, FFTMECH_K_OTHER, launch_set_masked(NB, mask, cD, c, em.st));
  CK(cudaMemcpyAsync(ctx->cn, c, sizeof(double) * NB, cudaMemcpyDeviceToDevice, em.st));
  op.c0c = 1.0 / dt;
  op.srcd = ctx->cn;
  op.src_scale = 1.0 / dt;
  op.mask = mask;
  sp.m0 = 1.0 / dt;
  sp.m1b = ctx->m1b;
  RC(emit_pcg<T, 1>(em, op, c, sp));
  return rec_end(em, SK_DIFF);
}

template <typename T>
fftmech_status enqueue_phasefield(Emit& em, const T* strain, const T* eig, const uint8_t* phase, T* H, double* d) {
  fftmech_ctx* ctx = em.ctx;
  em.sk = SK_PF;
  RC(rec_begin(em, SK_PF));
  const int B = ctx->B;
  Op<T> op;
  base_op<T>(ctx, op, phase);
  const double a = ctx->mat.Gc / (2.0 * ctx->mat.l0);
  const double b = ctx->mat.Gc * ctx->mat.l0 / 2.0;
  // history update; m0b[p] = a + mean(H) of each problem (on device)
  if (ctx->dim == 3)
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch3_history<T>(ctx->N, B, phase, op.lam[0], op.lam[1], op.mu[0], op.mu[1],
                                                      strain, eig, H, ctx->Hd, a, ctx->m0b, ctx->partials, ctx->sc,
                                                      em.st));
  else
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch_history<T>(ctx->N, B, phase, op.lam[0], op.lam[1], op.mu[0], op.mu[1],
                                                     strain, eig, H, ctx->Hd, a, ctx->m0b, ctx->partials, ctx->sc,
                                                     em.st));
  op.kap[0] = op.kap[1] = b;
  op.c0c = a;
  op.c0f = H;
  op.srcd = ctx->Hd;
  op.src_scale = 1.0;
  Spec<T> sp{};
  sp.m0b = ctx->m0b;
  sp.m1 = b / (ctx->h * ctx->h);
  RC(emit_pcg<T, 1>(em, op, d, sp));
  EM_LAUNCH(em, FFTMECH_K_OTHER, launch_pf_stats(ctx->N, B, phase, d, ctx->partials, res_dev(ctx, SK_PF), ctx->sc,
                                                 0.0, 0.0, 0.0, nullptr, em.st));
  return rec_end(em, SK_PF);
}

// Device pointers of one staggered step (after staging).
struct StepPtrs {
  const uint8_t* phase;
  double* c;
  void* cppt;
  void* eig;
  double* u;
  void* strain;
  void* stress;
  void* H;
  double* d;
  const uint8_t* mask;
  const void* eigf;
};

// One staggered step in Algorithm 1's order (Sec. 2.5).
template <typename T>
fftmech_status enqueue_step(Emit& em, const StepPtrs& s, const fftmech_step_params* prm) {
  fftmech_ctx* ctx = em.ctx;
  const size_t N = (size_t)ctx->N * ctx->B;
  // 1. diffusion of chemical species
  if (prm->diffusion_mode != FFTMECH_DIFF_NONE)
    RC(enqueue_diffusion<T>(em, s.phase, prm->diffusion_mode, prm->grad_c_mac, prm->c_macro, prm->dt, s.mask,
                            prm->dirichlet_value, s.c, prm->grad_c_mac_each, prm->c_macro_each));
  // 2. precipitation and eigenstrain
  if (prm->eig_mode == FFTMECH_EIG_FROM_PRECIPITATE)
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch_precipitate<T>(N, s.phase, s.c, ctx->mat.S_sol, ctx->mat.M_ppt, (T*)s.cppt,
                                                         (T*)s.eig, em.st));
  else
    EM_LAUNCH(em, FFTMECH_K_OTHER, launch_scale_copy<T>(N, (const T*)s.eigf, prm->eig_scale, (T*)s.eig, em.st));
  // 3. equilibrium with the stiffness degraded by the current damage
  RC(enqueue_equilibrium<T>(em, s.phase, (const T*)s.eig, s.d, prm->eps_mac, s.u, (T*)s.strain, (T*)s.stress));
  // 4. history and phase field
  RC(enqueue_phasefield<T>(em, (const T*)s.strain, (const T*)s.eig, s.phase, (T*)s.H, s.d));
  return FFTMECH_OK;
}

// ---------------------------------------------------------------- reports (host)
fftmech_solve_info& info_at(fftmech_solve_info* info, int b, int stride) { return info[(size_t)b * stride]; }

// Fills the records of solve `kind` (problem b at info[b * stride]) from the
// pinned copy of the record block; returns the first non-OK status.
fftmech_status collect(fftmech_ctx* ctx, int kind, fftmech_solve_info* info, int stride) {
  const SolverScalars* S = reinterpret_cast<const SolverScalars*>(ctx->h_rec + rec_sc_off(ctx, kind));
  const double* R = reinterpret_cast<const double*>(ctx->h_rec + rec_res_off(ctx, kind));
  const unsigned long long* t = reinterpret_cast<const unsigned long long*>(ctx->h_rec + rec_stamp_off(ctx, kind));
  const double ms = t[1] >= t[0] ? (double)(t[1] - t[0]) * 1e-6 : 0.0;
  const double N = (double)ctx->N;
  const bool three = ctx->dim == 3;
  fftmech_status worst = FFTMECH_OK;
  for (int b = 0; b < ctx->B; ++b) {
    const SolverScalars& f = S[b];
    fftmech_solve_info& i = info_at(info, b, stride);
    i.iters = f.iter;
    i.status = f.done ? f.status : FFTMECH_ERR_NOT_CONVERGED;
    i.rel_res = f.rz0 > 0 ? std::sqrt(std::max(f.rz, 0.0) / f.rz0) : 0.0;
    i.true_rel_res = f.rz0 > 0 ? std::sqrt(std::max(f.rz_true, 0.0) / f.rz0) : 0.0;
    i.device_ms = ms;
    if (kind == SK_EQ) {
      const int nv = nvoigt(ctx);
      const double* r = R + b * (2 * nv + 1);
      const double vox = three ? ctx->h * ctx->h * ctx->h : ctx->h * ctx->h;
      for (int k = 0; k < nv; ++k) {
        i.mean_stress[k] = r[k] / N;
        i.mean_strain[k] = r[nv + k] / N;
      }
      i.elastic_energy = r[2 * nv] * vox;
    } else if (kind == SK_DIFF) {
      if (ctx->last.diff_mode == FFTMECH_DIFF_HOMOGENISE) {
        const int nr = three ? 7 : 6, nd = three ? 3 : 2;
        const double* r = R + b * nr;
        for (int k = 0; k < nd; ++k) i.mean_flux[k] = r[2 + k];
        i.porosity = r[2 + nd];
        i.mean_c = r[3 + nd];
      } else {
        i.porosity = 1.0 - R[b * 3 + 2] / N;
      }
    } else {
      const double* r = R + b * 3;
      i.total_damage = r[0];
      i.frac_damaged = r[2] > 0 ? r[1] / r[2] : 0.0;
    }
    if (i.status != FFTMECH_OK && worst == FFTMECH_OK) worst = (fftmech_status)i.status;
  }
  return worst;
}

bool is_hard_error(fftmech_status s) {
  return s == FFTMECH_ERR_CUDA || s == FFTMECH_ERR_OOM || s == FFTMECH_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- running an operation
template <typename A>
void key_add(std::vector<unsigned char>& k, const A& a) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&a);
  k.insert(k.end(), p, p + sizeof(A));
}

// Captures `enqueue` into a graph and makes (or updates) the cached
// executable graph of operation `opk`.
template <typename F>
fftmech_status build_graph(fftmech_ctx* ctx, GraphCache& c, const std::vector<unsigned char>& key, F&& enqueue) {
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
  LaunchCount lc;
  Emit em = eager_emit(ctx);
  em.graph = true;
  em.lc = &lc;
  cudaStreamCaptureStatus cs;
  fftmech_status rc = FFTMECH_OK;
  if (cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &em.g, nullptr, nullptr, nullptr) != cudaSuccess)
    rc = set_err(ctx, FFTMECH_ERR_CUDA, "cudaStreamGetCaptureInfo failed");
  if (rc == FFTMECH_OK) rc = enqueue(em);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  if (rc == FFTMECH_OK && e != cudaSuccess)
    rc = set_err(ctx, FFTMECH_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  if (rc != FFTMECH_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  if (c.exec) {
    cudaGraphExecUpdateResultInfo ri;
    if (cudaGraphExecUpdate(c.exec, graph, &ri) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(c.exec);
      c.exec = nullptr;
    }
  }
  cudaError_t ei = cudaSuccess;
  if (!c.exec) ei = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    c.exec = nullptr;
    cudaGetLastError();
    return set_err(ctx, FFTMECH_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
  }
  c.key = key;
  c.lc = lc;
  ctx->graph_builds += 1;
  return FFTMECH_OK;
}

// Runs operation `opk` on the context's stream: into the caller's graph when
// the stream is being captured; as the cached graph (captured again when
// the arguments changed) by default; host-driven when asked for, while
// profiling, or after a graph failed (the reason is kept in graph_err).
// Returns without synchronising.
template <typename F>
fftmech_status run_op(fftmech_ctx* ctx, int opk, const std::vector<unsigned char>& key, F&& enqueue) {
  ctx->pending_lc = nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    Emit em = eager_emit(ctx);
    em.graph = true;
    CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &em.g, nullptr, nullptr, nullptr));
    return enqueue(em);
  }
  if (ctx->opts.execution == FFTMECH_EXEC_GRAPH && !ctx->prof && !ctx->graph_off) {
    GraphCache& c = ctx->gc[opk];
    fftmech_status rc = FFTMECH_OK;
    if (!c.exec || c.key != key) rc = build_graph(ctx, c, key, enqueue);
    if (rc == FFTMECH_OK) {
      const cudaError_t e = cudaGraphLaunch(c.exec, ctx->stream);
      if (e == cudaSuccess) {
        ctx->graph_launches += 1;
        ctx->pending_lc = &c.lc;
        return FFTMECH_OK;
      }
      cudaGetLastError();
      set_err(ctx, FFTMECH_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    }
    if (is_hard_error(rc) && rc != FFTMECH_ERR_CUDA) return rc;  // an argument error, not the graph
    // the graph path failed: remember why and continue host-driven
    snprintf(ctx->graph_err, sizeof(ctx->graph_err), "%s", ctx->err);
    ctx->err[0] = 0;
    ctx->graph_off = true;
  }
  Emit em = eager_emit(ctx);
  return enqueue(em);
}

// After the operation: wait for it, then report.
fftmech_status finish_sync(fftmech_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return FFTMECH_OK;
}

// Kernels run by the graph replay of the last operation, from its records:
// a solve's loop body ran once per iteration (the largest count of the batch),
// the replacement residual once per scheduled replacement, the outer body
// once plus once per restart.
void count_graph_kernels(fftmech_ctx* ctx) {
  const LaunchCount* lc = ctx->last.lc;
  if (!lc) return;
  long long n = lc->fixed;
  for (int k = 0; k < SK_COUNT; ++k) {
    if (!ctx->last.ran[k]) continue;
    const SolverScalars* S = reinterpret_cast<const SolverScalars*>(ctx->h_rec + rec_sc_off(ctx, k));
    long long it = 0, rep = 0, rst = 0;
    for (int b = 0; b < ctx->B; ++b) {
      it = std::max<long long>(it, S[b].iter);
      rep = std::max<long long>(rep, S[b].nreplace);
      rst = std::max<long long>(rst, S[b].nrestart);
    }
    // rounds: one plus one per replacement and per restart; the gate's
    // true-residual body once plus once per restart
    n += lc->body[k][LF_OUTER] * (1 + rep + rst) + lc->body[k][LF_LOOP] * std::max(0LL, it - rep) +
         lc->body[k][LF_REPLACE] * rep + lc->body[k][LF_GATE] * (1 + rst) + lc->body[k][LF_RESTART] * rst;
  }
  ctx->graph_kernels += n;
  ctx->last.lc = nullptr;
}

bool opts_ok(const fftmech_solver_opts* o) {
  return o->tol >= 0 && o->max_iter >= 0 && o->launch_mode >= 0 && o->launch_mode <= 3 &&
         (o->execution == FFTMECH_EXEC_GRAPH || o->execution == FFTMECH_EXEC_HOST) &&
         (o->precond == FFTMECH_PRECOND_LAPLACE || o->precond == FFTMECH_PRECOND_REFERENCE);
}

// Staged device pointers of a staggered step; `all_device`: nothing was
// staged (every pointer is device memory).
fftmech_status stage_step(fftmech_ctx* ctx, const fftmech_state* state, const fftmech_step_params* prm, StepPtrs& d,
                          bool& all_device) {
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  void *dphase, *dc, *dcppt, *deig, *du, *dstrain, *dstress, *dH, *dd, *dmask = nullptr, *deigf = nullptr;
  RC(stage_in(ctx, ST_PHASE, state->phase, N, true, &dphase));
  RC(stage_in(ctx, ST_C, state->c, N * 8, true, &dc));
  RC(stage_in(ctx, ST_CPPT, state->c_ppt, N * es, true, &dcppt));
  RC(stage_in(ctx, ST_EIG, state->eig, N * es, true, &deig));
  RC(stage_in(ctx, ST_U, state->u, (size_t)ctx->dim * N * 8, true, &du));
  RC(stage_in(ctx, ST_STRAIN, state->strain, nv * N * es, true, &dstrain));
  RC(stage_in(ctx, ST_STRESS, state->stress, nv * N * es, true, &dstress));
  RC(stage_in(ctx, ST_H, state->H, N * es, true, &dH));
  RC(stage_in(ctx, ST_DAMAGE, state->damage, N * 8, true, &dd));
  if (prm->diffusion_mode == FFTMECH_DIFF_TRANSIENT)
    RC(stage_in(ctx, ST_MASK, prm->dirichlet_mask, N, true, &dmask));
  if (prm->eig_mode == FFTMECH_EIG_PRESCRIBED) RC(stage_in(ctx, ST_EIGFIELD, prm->eig_field, N * es, true, &deigf));
  d = StepPtrs{(const uint8_t*)dphase, (double*)dc, dcppt, deig, (double*)du, dstrain, dstress, dH,
               (double*)dd, (const uint8_t*)dmask, deigf};
  all_device = dphase == state->phase && dc == state->c && dcppt == state->c_ppt && deig == state->eig &&
               du == state->u && dstrain == state->strain && dstress == state->stress && dH == state->H &&
               dd == state->damage && dmask == (const void*)prm->dirichlet_mask && deigf == prm->eig_field;
  return FFTMECH_OK;
}

fftmech_status check_step_args(fftmech_ctx* ctx, const fftmech_state* state, const fftmech_step_params* prm) {
  if (!state || !prm || !state->phase || !state->c || !state->eig || !state->u || !state->strain || !state->stress ||
      !state->H || !state->damage)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (prm->diffusion_mode != FFTMECH_DIFF_NONE && prm->diffusion_mode != FFTMECH_DIFF_HOMOGENISE &&
      prm->diffusion_mode != FFTMECH_DIFF_TRANSIENT)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "diffusion mode %d", prm->diffusion_mode);
  if (prm->diffusion_mode == FFTMECH_DIFF_TRANSIENT && !(prm->dt > 0))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt must be > 0 for TRANSIENT");
  if (prm->eig_mode == FFTMECH_EIG_PRESCRIBED && !prm->eig_field)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "eig_field is required for PRESCRIBED");
  if (prm->eig_mode != FFTMECH_EIG_PRESCRIBED && prm->eig_mode != FFTMECH_EIG_FROM_PRECIPITATE)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "eigenstrain mode %d", prm->eig_mode);
  for (const double* p : {prm->c_macro_each, prm->grad_c_mac_each})
    if (p && !is_device_ptr(p))
      return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "c_macro_each / grad_c_mac_each must be device memory");
  return FFTMECH_OK;
}

// Enqueues one staggered step on device pointers (graph or host-driven);
// with a bar, framed by the bar's element inputs and nodal update.
fftmech_status step_enqueue(fftmech_ctx* ctx, const StepPtrs& d, const fftmech_step_params* prm,
                            const BarDev* bar = nullptr) {
  std::vector<unsigned char> key;
  key_add(key, d);
  key_add(key, *prm);
  key_add(key, ctx->opts);
  if (bar) key_add(key, *bar);
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  RC(run_op(ctx, bar ? OP_BAR : OP_STEP, key, [&](Emit& em) -> fftmech_status {
    if (bar) EM_LAUNCH(em, FFTMECH_K_OTHER, launch_bar_inputs(bar->M, bar->dX, bar->c, bar->cbar, bar->G, em.st));
    RC(fp64 ? enqueue_step<double>(em, d, prm) : enqueue_step<float>(em, d, prm));
    if (bar)
      EM_LAUNCH(em, FFTMECH_K_OTHER, launch_bar_update(bar->M, bar->dX, bar->dt, bar->flux_in, bar->c,
                                                       res_dev(ctx, SK_DIFF), ctx->dim == 3 ? 7 : 6, em.st));
    return rec_publish(em);
  }));
  ctx->last = LastOp();
  ctx->last.valid = 1;
  ctx->last.ran[SK_DIFF] = prm->diffusion_mode != FFTMECH_DIFF_NONE;
  ctx->last.ran[SK_EQ] = ctx->last.ran[SK_PF] = 1;
  ctx->last.diff_mode = prm->diffusion_mode;
  ctx->last.c_macro = prm->c_macro;
  ctx->last.lc = ctx->pending_lc;
  return FFTMECH_OK;
}

// Fills info[3 B] from the records of the last staggered step (the stream
// has been synchronised).
fftmech_status step_collect(fftmech_ctx* ctx, fftmech_solve_info* info) {
  count_graph_kernels(ctx);
  std::memset(info, 0, sizeof(fftmech_solve_info) * 3 * ctx->B);
  fftmech_status worst = FFTMECH_OK;
  for (int k = 0; k < SK_COUNT; ++k) {
    if (!ctx->last.ran[k]) continue;
    const fftmech_status s = collect(ctx, k, info + k, 3);
    if (s != FFTMECH_OK && worst == FFTMECH_OK) worst = s;
  }
  return worst;
}

// ---------------------------------------------------------------- adjoint
// Device buffers of one adjoint call, freed together.
struct DevBuffers {
  std::vector<void*> ptrs;
  bool ok = true;
  template <typename P>
  P* get(size_t bytes) {
    void* p = nullptr;
    if (!ok || cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<P*>(p);
  }
  ~DevBuffers() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// Solver status of the last solve on the context (one problem).
fftmech_status last_solve_status(fftmech_ctx* ctx, cudaStream_t st) {
  SolverScalars h;
  CK(cudaMemcpyAsync(&h, ctx->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!h.done) return FFTMECH_ERR_NOT_CONVERGED;
  return (fftmech_status)h.status;
}

// Forward with checkpoints (H, d, u every k steps), then per segment from
// the last: recompute its steps from the checkpoint keeping strain, H and d
// of each, and run the reverse steps (phase-field adjoint PCG, history /
// psi+ kernel, equilibrium adjoint PCG with the prescribed-stress source,
// accumulation kernel).
template <typename T>
fftmech_status adjoint_impl(fftmech_ctx* ctx, const uint8_t* phase, const T* efield, int S, const double* ramp,
                            const double* E, int objective, int k, double* grad, double* J,
                            fftmech_solve_info* info_last) {
  cudaStream_t st = ctx->stream;
  const long long N = ctx->N;
  const int dim = ctx->dim, nv = nvoigt(ctx);
  const size_t es = sizeof(T);
  const int nck = (S + k - 1) / k;
  DevBuffers mem;
  double* c = mem.get<double>(N * 8);
  T* cppt = mem.get<T>(N * es);
  T* eig = mem.get<T>(N * es);
  double* u = mem.get<double>((size_t)dim * N * 8);
  T* strain = mem.get<T>((size_t)nv * N * es);
  T* stress = mem.get<T>((size_t)nv * N * es);
  T* H = mem.get<T>(N * es);
  double* d = mem.get<double>(N * 8);
  std::vector<T*> ckH(nck), segH(k), segS(k);
  std::vector<double*> ckd(nck), cku(nck), segd(k);
  for (int i = 0; i < nck; ++i) {
    ckH[i] = mem.get<T>(N * es);
    ckd[i] = mem.get<double>(N * 8);
    cku[i] = mem.get<double>((size_t)dim * N * 8);
  }
  for (int j = 0; j < k; ++j) {
    segH[j] = mem.get<T>(N * es);
    segd[j] = mem.get<double>(N * 8);
    segS[j] = mem.get<T>((size_t)nv * N * es);
  }
  T* tau = mem.get<T>((size_t)nv * N * es);
  double* dJde = mem.get<double>(N * 8);
  double* ddirect = mem.get<double>(N * 8);
  double* dJdd = mem.get<double>(N * 8);
  double* dJdH = mem.get<double>(N * 8);
  double* lampf = mem.get<double>(N * 8);
  double* mu = mem.get<double>((size_t)dim * N * 8);
  double* scl = mem.get<double>(4 * 8);  // [pf s, pf 1/s, eq s, eq 1/s]
  unsigned long long* mx = mem.get<unsigned long long>(2 * 8);
  if (!mem.ok) return set_err(ctx, FFTMECH_ERR_OOM, "adjoint buffers");
  CK(cudaMemsetAsync(c, 0, N * 8, st));
  CK(cudaMemsetAsync(u, 0, (size_t)dim * N * 8, st));
  CK(cudaMemsetAsync(H, 0, N * es, st));
  CK(cudaMemsetAsync(d, 0, N * 8, st));
  CK(cudaMemsetAsync(grad, 0, N * 8, st));
  fftmech_step_params prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.diffusion_mode = FFTMECH_DIFF_NONE;
  prm.eig_mode = FFTMECH_EIG_PRESCRIBED;
  prm.eig_field = efield;
  for (int i = 0; i < nv; ++i) prm.eps_mac[i] = E[i];
  const StepPtrs sp{phase, c, cppt, eig, u, strain, stress, H, d, nullptr, efield};
  auto step = [&](int s) -> fftmech_status {
    prm.eig_scale = ramp[s];
    RC(step_enqueue(ctx, sp, &prm));
    RC(finish_sync(ctx));
    return FFTMECH_OK;
  };
  // forward
  fftmech_status worst = FFTMECH_OK;
  std::vector<fftmech_solve_info> rec(3);
  for (int s = 0; s < S; ++s) {
    if (s % k == 0) {
      const int i = s / k;
      CK(cudaMemcpyAsync(ckH[i], H, N * es, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ckd[i], d, N * 8, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(cku[i], u, (size_t)dim * N * 8, cudaMemcpyDeviceToDevice, st));
    }
    RC(step(s));
    const fftmech_status ws = step_collect(ctx, rec.data());
    if (ws != FFTMECH_OK && worst == FFTMECH_OK) worst = ws;
  }
  if (info_last) std::memcpy(info_last, rec.data(), sizeof(fftmech_solve_info) * 3);
  *J = objective == FFTMECH_OBJ_ENERGY ? rec[1].elastic_energy : rec[2].total_damage;
  // reverse
  double lam0, mu0, lam1, mu1;
  lame(ctx->mat.E_pore, ctx->mat.nu_pore, lam0, mu0);
  lame(ctx->mat.E_solid, ctx->mat.nu_solid, lam1, mu1);
  const double a = ctx->mat.Gc / (2.0 * ctx->mat.l0), b = ctx->mat.Gc * ctx->mat.l0 / 2.0;
  const double vol = dim == 3 ? ctx->h * ctx->h * ctx->h : ctx->h * ctx->h;
  // Right-hand sides normalised to the forward solves' magnitudes: a stress
  // at strain 1e-3 (equilibrium) and the energy density at that strain
  // (phase field), from the solid's stiffness.
  const double m_solid = lam1 + 2.0 * mu1;
  const double target_eq = 1e-3 * m_solid, target_pf = 0.5e-6 * m_solid;
  CK(cudaMemsetAsync(dJdH, 0, N * 8, st));
  CK(launch_fill(N, objective == FFTMECH_OBJ_DAMAGE ? 1.0 : 0.0, dJdd, st));
  Emit em = eager_emit(ctx);
  auto track = [&](fftmech_status s2) {
    if (s2 != FFTMECH_OK && worst == FFTMECH_OK) worst = s2;
  };
  for (int seg = nck - 1; seg >= 0; --seg) {
    const int s0 = seg * k, s1 = std::min(S, s0 + k);
    CK(cudaMemcpyAsync(H, ckH[seg], N * es, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d, ckd[seg], N * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(u, cku[seg], (size_t)dim * N * 8, cudaMemcpyDeviceToDevice, st));
    for (int s = s0; s < s1; ++s) {
      RC(step(s));
      const int j = s - s0;
      CK(cudaMemcpyAsync(segS[j], strain, (size_t)nv * N * es, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(segH[j], H, N * es, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(segd[j], d, N * 8, cudaMemcpyDeviceToDevice, st));
    }
    for (int s = s1 - 1; s >= s0; --s) {
      const int j = s - s0;
      const T* Hprev = j > 0 ? segH[j - 1] : ckH[seg];
      const double* dprev = j > 0 ? segd[j - 1] : ckd[seg];
      // phase-field adjoint: A(H_s) lambda = dJ/dd_s
      CK(launch_adj_m0b<T>(N, segH[j], a, ctx->m0b, st));
      {
        Op<T> op;
        base_op<T>(ctx, op, phase);
        op.kap[0] = op.kap[1] = b;
        op.c0c = a;
        op.c0f = segH[j];
        op.srcd = dJdd;
        op.src_scale = 1.0;
        Spec<T> spec{};
        spec.m0b = ctx->m0b;
        spec.m1 = b / (ctx->h * ctx->h);
        CK(cudaMemsetAsync(lampf, 0, N * 8, st));
        CK(launch_adj_normalise<double>(N, dJdd, mx, target_pf, scl, st));
        RC(emit_pcg<T, 1>(em, op, lampf, spec));
        track(last_solve_status(ctx, st));
      }
      CK(launch_adj_history<T>(dim, N, phase, lam0, lam1, mu0, mu1, segS[j], efield, ramp[s], Hprev, segd[j], lampf,
                               scl + 1, dJdH, tau, dJde, ddirect, objective == FFTMECH_OBJ_ENERGY && s == S - 1 ? 1 : 0,
                               dprev, ctx->mat.kappa, vol, st));
      // equilibrium adjoint: K(d_{s-1}) mu = grad+^T tau
      CK(launch_degradation<T>(N, dprev, ctx->mat.kappa, (T*)ctx->g, st));
      {
        Op<T> op;
        base_op<T>(ctx, op, phase);
        op.g = (const T*)ctx->g;
        op.pre = tau;
        Spec<T> spec{};
        spec.m0 = 0.0;
        spec.m1 = 1.0 / (ctx->h * ctx->h);
        CK(cudaMemsetAsync(mu, 0, (size_t)dim * N * 8, st));
        CK(launch_adj_normalise<T>((long long)nv * N, tau, mx + 1, target_eq, scl + 2, st));
        RC(dim == 3 ? emit_pcg<T, 3>(em, op, mu, spec) : emit_pcg<T, 2>(em, op, mu, spec));
        track(last_solve_status(ctx, st));
      }
      CK(launch_adj_eqpost<T>(dim, ctx->nx, ctx->ny, ctx->nz, phase, lam0, lam1, mu0, mu1, segS[j], efield, ramp[s],
                              dprev, ctx->mat.kappa, mu, scl + 3, ctx->h, dJde, ddirect, dJdd, grad, st));
    }
  }
  CK(cudaStreamSynchronize(st));
  return worst;
}

// ---------------------------------------------------------------- launch-shape autotuning
// Choices of the tunable launch shapes of a context, cached for the process
// per (device, dimension, grid, batch, precision).
struct TuneChoice {
  int L_dir, L_upd, ty, zc, grid, cols, L_ds;
};
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
struct TuneEntry {
  TuneChoice choice;
  double before_us, after_us;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

TuneKey tune_key(const fftmech_ctx* ctx) {
  return TuneKey(ctx->device, ctx->dim, ctx->nx, ctx->ny, ctx->nz, ctx->B, (int)ctx->prec);
}

TuneChoice current_choice(const fftmech_ctx* ctx) {
  return TuneChoice{ctx->lshape.L_dir, ctx->lshape.L_upd, ctx->sshape.ty, ctx->sshape.zc, ctx->sshape.grid,
                    ctx->shape.cols, ds_active(ctx) ? ctx->lshape.L_ds : 0};
}

// The column strip width's thread count and shared memory (2D).
template <typename T>
bool cols_ok(const fftmech_ctx* ctx, int cw) {
  const int ny = ctx->ny;
  const bool fixed = sizeof(T) == 4 && (ny == 81 || ny == 243 || ny == 729 || ny == 2187 || ny == 128 || ny == 256 ||
                                        ny == 512 || ny == 1024);
  if (fixed && cw != 2 && cw != 4 && cw != 8) return false;
  const size_t smem = (size_t)ny * cw * sizeof(cx<T>) + tw_smem_bytes<T>(ny) + (size_t)(ny + cw) * sizeof(T);
  return cw >= 1 && smem <= ctx->optin - 1024 && (fixed || need_threads(ctx->py, cw) <= 512) &&
         (size_t)ctx->B * ctx->nx >= (size_t)1;
}

template <typename T>
bool choice_ok(const fftmech_ctx* ctx, const TuneChoice& c) {
  const int spec3 = ctx->dim == 3 ? (int)nxs_of(ctx->nx, 3) : ctx->nx;
  if (!line_shape_ok<T>(ctx->px, c.L_dir, true, ctx->dim, spec3, ctx->optin)) return false;
  if (!line_shape_ok<T>(ctx->px, c.L_upd, false, ctx->dim, spec3, ctx->optin)) return false;
  if (c.L_dir > ctx->ny * ctx->nz || c.L_upd > ctx->ny * ctx->nz || c.grid < 1) return false;
  if (c.L_ds != 0 && (ctx->dim != 2 || !ds_shape_ok<T>(ctx->px, c.L_ds, ctx->ny, ctx->optin))) return false;
  if (ctx->dim == 2) return (c.ty == 4 || c.ty == 8) && cols_ok<T>(ctx, c.cols);
  return c.ty == 4 && c.zc >= 1 && c.zc <= std::min(16, ctx->nz);
}

// Applies a choice; the cached graphs embed the old shapes and are dropped.
template <typename T>
void apply_choice(fftmech_ctx* ctx, const TuneChoice& c) {
  ctx->lshape.L_dir = c.L_dir;
  ctx->lshape.thr_dir = line_threads(ctx->px, c.L_dir, ctx->dim);
  ctx->lshape.L_upd = c.L_upd;
  ctx->lshape.thr_upd = line_threads(ctx->px, c.L_upd, ctx->dim);
  if (c.L_ds > 0) {
    ctx->lshape.L_ds = c.L_ds;
    ctx->lshape.thr_ds = ds_threads(ctx->px, c.L_ds);
  }
  ctx->ds_choice = c.L_ds > 0 ? 1 : 0;
  ctx->sshape.ty = c.ty;
  ctx->sshape.zc = c.zc;
  ctx->sshape.grid = c.grid;
  if (ctx->dim == 2 && c.cols != ctx->shape.cols) {
    ctx->shape.cols = c.cols;
    const int ny = ctx->ny;
    const bool fixed = sizeof(T) == 4 && (ny == 81 || ny == 243 || ny == 729 || ny == 2187 || ny == 128 ||
                                          ny == 256 || ny == 512 || ny == 1024);
    ctx->shape.threads_col = fixed ? (c.cols >= 4 ? 512 : 256)
                                   : std::min(512, std::max(128, round32(need_threads(ctx->py, c.cols))));
  }
  for (GraphCache& g : ctx->gc) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
  }
}

// Time of `iterations` equilibrium PCG iterations (graph execution, the
// iterate reset to zero first), best of two after one warm-up.
template <typename T>
fftmech_status time_solve(fftmech_ctx* ctx, const uint8_t* phase, const T* eig, double* u, double* ms_out) {
  const double E[6] = {0, 0, 0, 0, 0, 0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  fftmech_status rc = FFTMECH_OK;
  for (int rep = 0; rep < 3 && rc == FFTMECH_OK; ++rep) {
    if (cudaMemsetAsync(u, 0, sizeof(double) * ctx->dim * ctx->N * ctx->B, ctx->stream) != cudaSuccess) {
      rc = FFTMECH_ERR_CUDA;
      break;
    }
    std::vector<unsigned char> key;
    key_add(key, phase);
    key_add(key, u);
    cudaEventRecord(e0, ctx->stream);
    rc = run_op(ctx, OP_EQ, key, [&](Emit& em) -> fftmech_status {
      RC(enqueue_equilibrium<T>(em, phase, eig, nullptr, E, u, nullptr, nullptr));
      return rec_publish(em);
    });
    cudaEventRecord(e1, ctx->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = FFTMECH_ERR_CUDA;
    float ms = 0.f;
    if (rc == FFTMECH_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FFTMECH_ERR_CUDA;
    if (rep > 0) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  *ms_out = best;
  return rc;
}

template <typename T>
fftmech_status autotune_impl(fftmech_ctx* ctx, int iterations, double* before_us, double* after_us) {
  const size_t NB = (size_t)ctx->N * ctx->B;
  // synthetic two-phase microstructure (70 % solid, hashed voxel pattern)
  // with a pore eigenstrain: the kernels' cost does not depend on the data
  std::vector<uint8_t> hphase(NB);
  std::vector<T> heig(NB);
  for (size_t i = 0; i < NB; ++i) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z ^= z >> 31;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 29;
    hphase[i] = (z % 10) < 7 ? 1 : 0;
    heig[i] = hphase[i] ? T(0) : T(1e-3);
  }
  uint8_t* phase = nullptr;
  T* eig = nullptr;
  double* u = nullptr;
  auto release = [&]() {
    if (phase) cudaFree(phase);
    if (eig) cudaFree(eig);
    if (u) cudaFree(u);
  };
  if (cudaMalloc((void**)&phase, NB) != cudaSuccess || cudaMalloc((void**)&eig, NB * sizeof(T)) != cudaSuccess ||
      cudaMalloc((void**)&u, NB * ctx->dim * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return set_err(ctx, FFTMECH_ERR_OOM, "autotune buffers");
  }
  if (cudaMemcpy(phase, hphase.data(), NB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(eig, heig.data(), NB * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    release();
    return set_err(ctx, FFTMECH_ERR_CUDA, "autotune buffers");
  }
  const fftmech_solver_opts saved = ctx->opts;
  const bool saved_off = ctx->graph_off;
  ctx->opts.tol = 0.0;
  ctx->opts.max_iter = iterations;
  ctx->opts.execution = FFTMECH_EXEC_GRAPH;
  TuneChoice best = current_choice(ctx);
  double best_ms = 0.0;
  fftmech_status rc = time_solve<T>(ctx, phase, eig, u, &best_ms);
  const double first_ms = best_ms;
  auto consider = [&](TuneChoice c) {
    if (rc != FFTMECH_OK || !choice_ok<T>(ctx, c)) return;
    apply_choice<T>(ctx, c);
    double ms = 0.0;
    rc = time_solve<T>(ctx, phase, eig, u, &ms);
    if (rc == FFTMECH_OK && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    apply_choice<T>(ctx, best);
  };
  // coordinate descent: one parameter at a time, each from the best so far
  if (ctx->dim == 2) {
    for (int cw : {4, 8, ctx->shape.cols / 2, ctx->shape.cols * 2}) {
      TuneChoice c = best;
      if (cw == best.cols || cw < 1) continue;
      c.cols = cw;
      consider(c);
    }
    {
      TuneChoice c = best;
      c.ty = best.ty == 8 ? 4 : 8;
      consider(c);
    }
  } else {
    for (int zc : {2, 4, 8, 16}) {
      TuneChoice c = best;
      if (zc == best.zc) continue;
      c.zc = zc;
      consider(c);
    }
  }
  for (int f : {2, -2}) {
    TuneChoice c = best;
    c.grid = f > 0 ? best.grid * 2 : std::max(1, best.grid / 2);
    if (c.grid != best.grid) consider(c);
  }
  for (int which = 0; which < 2; ++which) {
    const int L0 = which == 0 ? best.L_dir : best.L_upd;
    for (int L : {L0 / 2, L0 * 2, L0 + 1, L0 - 1}) {
      TuneChoice c = best;
      if (L < 1 || L == L0) continue;
      (which == 0 ? c.L_dir : c.L_upd) = L;
      consider(c);
    }
  }
  // split or fused direction and stencil (2D grids where the iteration is
  // latency-bound): the rule's rows per block, then its neighbours
  if (ctx->dim == 2 && ctx->ds_rule > 0 && (long long)ctx->N * ctx->B <= (1LL << 21)) {
    const int L0 = best.L_ds > 0 ? best.L_ds : ctx->ds_rule;
    for (int L : {0, L0, L0 / 2, L0 * 2, L0 + 1, L0 - 1}) {
      TuneChoice c = best;
      if (L < 0 || L == best.L_ds) continue;
      c.L_ds = L;
      consider(c);
    }
  }
  ctx->opts = saved;
  ctx->graph_off = saved_off;
  apply_choice<T>(ctx, best);
  release();
  if (rc != FFTMECH_OK) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[tune_key(ctx)] = TuneEntry{best, 1e3 * first_ms / iterations, 1e3 * best_ms / iterations};
  }
  if (before_us) *before_us = 1e3 * first_ms / iterations;
  if (after_us) *after_us = 1e3 * best_ms / iterations;
  snprintf(ctx->tune_desc, sizeof(ctx->tune_desc), "L_dir=%d L_upd=%d ty=%d zc=%d grid=%d cols=%d L_ds=%d",
           best.L_dir, best.L_upd, best.ty, best.zc, best.grid, best.cols, best.L_ds);
  return FFTMECH_OK;
}

}  // namespace

// Unnormalised in-place transform of an nz x ny x nx complex array (x
// fastest) on `st`: x lines, then the y columns of every plane, then the z
// columns (the array seen as nz rows of nx ny points). Plans are cached for
// the process. Enqueues only.
fftmech_status fft_inplace(int nx, int ny, int nz, bool fp64, bool inverse, void* data, cudaStream_t st) {
  fftmech_ctx* ctx = nullptr;  // for CK's error path (no message storage)
  if (!factor_ok(nx) || !factor_ok(ny) || !factor_ok(nz) || nx < 2) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  HostPlan px, py, pz;
  if (cached_plan(dev, nx, px) != cudaSuccess || cached_plan(dev, ny, py) != cudaSuccess ||
      cached_plan(dev, nz, pz) != cudaSuccess) {
    cudaGetLastError();
    return FFTMECH_ERR_OOM;
  }
  const int nsm = prop.multiProcessorCount;
  const size_t optin = prop.sharedMemPerBlockOptin;
  Shape2 sh{}, shz{};
  bool shp = fp64 ? choose_shape_fft<double>(px, py, nsm, optin, sh) : choose_shape_fft<float>(px, py, nsm, optin, sh);
  if (shp && nz > 1)
    shp = fp64 ? choose_shape_fft<double>(px, pz, nsm, optin, shz) : choose_shape_fft<float>(px, pz, nsm, optin, shz);
  if (!shp) return FFTMECH_ERR_UNSUPPORTED_SIZE;
  sh.batch = nz;  // the y pass runs plane by plane (grid.y = plane)
  shz.batch = 1;
  const int inv = inverse ? 1 : 0;
  auto run = [&](auto zero) -> cudaError_t {
    using T = decltype(zero);
    Spec<T> sp{};
    cudaError_t e = launch_rowfft_f<T>(px.fam, nx, ny * nz, (cx<T>*)data, dev_plan<T>(px), inv, sh, st);
    if (e == cudaSuccess && ny > 1)
      e = launch_colpass_f<T>(py.fam, nx, ny, (cx<T>*)data, dev_plan<T>(py), sp, sh, COL_PLAIN, inv, nullptr,
                              nullptr, nullptr, st);
    if (e == cudaSuccess && nz > 1)
      e = launch_colpass_f<T>(pz.fam, nx * ny, nz, (cx<T>*)data, dev_plan<T>(pz), sp, shz, COL_PLAIN, inv, nullptr,
                              nullptr, nullptr, st);
    return e;
  };
  const cudaError_t e = fp64 ? run(0.0) : run(0.0f);
  return e == cudaSuccess ? FFTMECH_OK : FFTMECH_ERR_CUDA;
}

// ---------------------------------------------------------------- gradient-operator variants
// Symbol D(k) of a gradient operator of Sec. 2.6 along an axis of n points
// (theta = 2 pi k / n): forward (e^{i theta} - 1) / h, central
// i sin(theta) / h, 8th-order central i sum_m 2 c_m sin(m theta) / h, Fourier
// i 2 pi k' / (n h) with k' folded to (-n/2, n/2].
std::vector<cx<double>> grad_symbol(int op, int n, double h) {
  // 8th-order central coefficients from the moment conditions
  // sum_m 2 m^(2j - 1) c_m = delta_j1, j = 1 .. 4 (Gaussian elimination)
  double c8[4] = {0, 0, 0, 0};
  if (op == FFTMECH_GRAD_CENTRAL8) {
    double A[4][5];
    for (int j = 0; j < 4; ++j) {
      for (int m = 0; m < 4; ++m) A[j][m] = 2.0 * std::pow((double)(m + 1), 2 * j + 1);
      A[j][4] = j == 0 ? 1.0 : 0.0;
    }
    for (int col = 0; col < 4; ++col) {
      int piv = col;
      for (int r = col + 1; r < 4; ++r)
        if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
      for (int k = 0; k < 5; ++k) std::swap(A[col][k], A[piv][k]);
      for (int r = 0; r < 4; ++r) {
        if (r == col) continue;
        const double f = A[r][col] / A[col][col];
        for (int k = col; k < 5; ++k) A[r][k] -= f * A[col][k];
      }
    }
    for (int m = 0; m < 4; ++m) c8[m] = A[m][4] / A[m][m];
  }
  std::vector<cx<double>> d(n);
  for (int k = 0; k < n; ++k) {
    const double th = 2.0 * M_PI * k / n;
    cx<double> v{0.0, 0.0};
    if (op == FFTMECH_GRAD_FORWARD) {
      v.re = (std::cos(th) - 1.0) / h;
      v.im = std::sin(th) / h;
    } else if (op == FFTMECH_GRAD_CENTRAL) {
      v.im = std::sin(th) / h;
    } else if (op == FFTMECH_GRAD_CENTRAL8) {
      double s = 0.0;
      for (int m = 0; m < 4; ++m) s += 2.0 * c8[m] * std::sin((m + 1) * th);
      v.im = s / h;
    } else {
      const int kf = k <= n / 2 ? k : k - n;
      v.im = 2.0 * M_PI * kf / (n * h);
    }
    d[k] = v;
  }
  return d;
}

// Homogenised diffusion (Eqs. diffusion, diffusion-final, phi-fft) with the
// gradient operator `op`: PCG on the spectral vector phi_hat (kernels in
// variants.cu), the operator applied through one inverse and one forward
// transform of the gradient per iteration, the preconditioner 1 / |D|^2.
// FP64; host-driven (the scalars are read every iteration).
fftmech_status homogenise_operator_impl(fftmech_ctx* ctx, const uint8_t* phase, int op, const double G[3],
                                        double* phi, double* gradc, fftmech_solve_info* info) {
  using cxd = cx<double>;
  cudaStream_t st = ctx->stream;
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz, dim = ctx->dim;
  const long long N = ctx->N;
  const size_t cb = (size_t)N * sizeof(cxd);
  DevBuffers mem;
  cxd* P = mem.get<cxd>(cb);
  cxd* R = mem.get<cxd>(cb);
  cxd* X = mem.get<cxd>(cb);
  cxd* Z = mem.get<cxd>(cb);
  cxd* Q = mem.get<cxd>(cb);
  cxd* W1 = mem.get<cxd>(cb);
  cxd* W2 = dim == 3 ? mem.get<cxd>(cb) : nullptr;
  cxd* dx = mem.get<cxd>((size_t)nx * sizeof(cxd));
  cxd* dy = mem.get<cxd>((size_t)ny * sizeof(cxd));
  cxd* dz = mem.get<cxd>((size_t)nz * sizeof(cxd));
  const int nb = var_dot_blocks(N);
  double* part = mem.get<double>((size_t)2 * nb * sizeof(double));
  if (!mem.ok) return set_err(ctx, FFTMECH_ERR_OOM, "operator-variant buffers");
  const double h = ctx->h_diff;
  const auto tx = grad_symbol(op, nx, h), ty = grad_symbol(op, ny, h), tz = grad_symbol(op, nz, h);
  CK(cudaMemcpyAsync(dx, tx.data(), nx * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dy, ty.data(), ny * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dz, tz.data(), nz * sizeof(cxd), cudaMemcpyHostToDevice, st));
  const VarGrid g{nx, ny, nz, dim, N, dx, dy, dz};
  const double invN = 1.0 / (double)N;
  const double kp = ctx->mat.D_pore, ks = ctx->mat.D_solid;
  const double zero[3] = {0, 0, 0};
  std::vector<double> hpart(2 * nb);
  auto fft = [&](cxd* a, bool inv) -> fftmech_status { return fft_inplace(nx, ny, nz, true, inv, a, st); };
  auto dot = [&](const cxd* a, const cxd* b, double& out) -> fftmech_status {
    CK(launch_var_dot(N, a, b, part, st));
    CK(cudaMemcpyAsync(hpart.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out = 0.0;
    for (int i = 0; i < nb; ++i) out += hpart[i];
    return FFTMECH_OK;
  };
  // q = s D^H F[kappa (F^-1(D p) / N + Gm)]; p = NULL: the gradient is 0
  auto apply = [&](const cxd* p, cxd* q, const double* Gm, double s) -> fftmech_status {
    if (p) {
      CK(launch_var_grad(g, p, W1, W2, st));
      RC(fft(W1, true));
      if (W2) RC(fft(W2, true));
    } else {
      CK(cudaMemsetAsync(W1, 0, cb, st));
      if (W2) CK(cudaMemsetAsync(W2, 0, cb, st));
    }
    CK(launch_var_flux(g, phase, kp, ks, Gm, invN, W1, W2, st));
    RC(fft(W1, false));
    if (W2) RC(fft(W2, false));
    CK(launch_var_div(g, W1, W2, s, q, st));
    return FFTMECH_OK;
  };
  RC(apply(nullptr, R, G, -1.0));  // f_hat = -D^H F[kappa G]
  CK(cudaMemsetAsync(X, 0, cb, st));
  CK(launch_var_precond(g, R, Z, st));
  CK(cudaMemcpyAsync(P, Z, cb, cudaMemcpyDeviceToDevice, st));
  double rz = 0.0;
  RC(dot(R, Z, rz));
  const double rz0 = rz;
  const double tol2 = ctx->opts.tol * ctx->opts.tol;
  int it = 0;
  fftmech_status status = FFTMECH_OK;
  while (rz0 > 0.0 && rz > tol2 * rz0) {
    if (it >= ctx->opts.max_iter) {
      status = FFTMECH_ERR_NOT_CONVERGED;
      break;
    }
    RC(apply(P, Q, zero, 1.0));
    double pq = 0.0;
    RC(dot(P, Q, pq));
    if (!(pq > 0.0) || !std::isfinite(pq)) {
      status = FFTMECH_ERR_NONFINITE;
      break;
    }
    const double alpha = rz / pq;
    CK(launch_var_axpy(N, alpha, P, Q, X, R, st));
    CK(launch_var_precond(g, R, Z, st));
    double rzn = 0.0;
    RC(dot(R, Z, rzn));
    ++it;
    CK(launch_var_dir(N, rzn / rz, Z, P, st));
    rz = rzn;
  }
  // phi = F^-1(phi_hat) / N; grad c = G + F^-1(D phi_hat) / N; <j> = -<kappa grad c>
  CK(cudaMemcpyAsync(W1, X, cb, cudaMemcpyDeviceToDevice, st));
  RC(fft(W1, true));
  if (phi) CK(launch_var_real(g, W1, nullptr, invN, phi, nullptr, nullptr, st));
  CK(launch_var_grad(g, X, W1, W2, st));
  RC(fft(W1, true));
  if (W2) RC(fft(W2, true));
  CK(launch_var_flux(g, phase, 1.0, 1.0, G, invN, W1, W2, st));  // grad c
  if (gradc)
    CK(launch_var_real(g, W1, W2, 1.0, gradc, dim >= 2 ? gradc + N : nullptr, dim == 3 ? gradc + 2 * N : nullptr,
                       st));
  CK(launch_var_flux(g, phase, kp, ks, zero, 1.0, W1, W2, st));  // kappa grad c
  double mean[3] = {0, 0, 0};
  for (int c = 0; c < (dim == 3 ? 2 : 1); ++c) {
    CK(launch_var_sum(N, c == 0 ? W1 : W2, part, st));
    CK(cudaMemcpyAsync(hpart.data(), part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
      a += hpart[2 * i];
      b += hpart[2 * i + 1];
    }
    if (c == 0) {
      mean[0] = -a * invN;
      mean[1] = -b * invN;
    } else {
      mean[2] = -a * invN;
    }
  }
  CK(cudaStreamSynchronize(st));
  std::memset(info, 0, sizeof(*info));
  info->status = status;
  info->iters = it;
  info->rel_res = rz0 > 0 ? std::sqrt(std::max(rz, 0.0) / rz0) : 0.0;
  info->true_rel_res = info->rel_res;
  for (int k = 0; k < dim; ++k) info->mean_flux[k] = mean[k];
  return status;
}

// Mechanical equilibrium with a chosen gradient operator (Sec. 2.6 applied
// to Eqs. solid and solid-final): the same spectral-operator PCG as the
// diffusion above, on the d displacement spectra, with the stress formed in
// real space from F^-1(sym D u). FP64, host-driven, one problem.
fftmech_status equilibrium_operator_impl(fftmech_ctx* ctx, const uint8_t* phase, const double* eig,
                                         const double* damage, const double E[6], int op, double* strain,
                                         double* stress, fftmech_solve_info* info) {
  using cxd = cx<double>;
  cudaStream_t st = ctx->stream;
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz, dim = ctx->dim;
  const long long N = ctx->N, nU = (long long)dim * N;
  const size_t cb = (size_t)N * sizeof(cxd), cu = (size_t)nU * sizeof(cxd);
  const VarElSpec spec = var_el_spec(dim);
  DevBuffers mem;
  cxd* P = mem.get<cxd>(cu);
  cxd* R = mem.get<cxd>(cu);
  cxd* X = mem.get<cxd>(cu);
  cxd* Z = mem.get<cxd>(cu);
  cxd* Q = mem.get<cxd>(cu);
  cxd* W[3] = {nullptr, nullptr, nullptr};
  for (int w = 0; w < spec.nw; ++w) W[w] = mem.get<cxd>(cb);
  cxd* dx = mem.get<cxd>((size_t)nx * sizeof(cxd));
  cxd* dy = mem.get<cxd>((size_t)ny * sizeof(cxd));
  cxd* dz = mem.get<cxd>((size_t)nz * sizeof(cxd));
  const int nb = var_dot_blocks(nU);
  const int nbs = var_dot_blocks(N);
  double* part = mem.get<double>((size_t)2 * std::max(nb, nbs) * sizeof(double));
  if (!mem.ok) return set_err(ctx, FFTMECH_ERR_OOM, "operator-variant buffers");
  const double h = ctx->h;
  const auto tx = grad_symbol(op, nx, h), ty = grad_symbol(op, ny, h), tz = grad_symbol(op, nz, h);
  CK(cudaMemcpyAsync(dx, tx.data(), nx * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dy, ty.data(), ny * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dz, tz.data(), nz * sizeof(cxd), cudaMemcpyHostToDevice, st));
  const VarGrid g{nx, ny, nz, dim, N, dx, dy, dz};
  const double invN = 1.0 / (double)N;
  double lam[2], mu[2];
  lame(ctx->mat.E_pore, ctx->mat.nu_pore, lam[0], mu[0]);
  lame(ctx->mat.E_solid, ctx->mat.nu_solid, lam[1], mu[1]);
  const double kappa = ctx->mat.kappa;
  const double zero[6] = {0, 0, 0, 0, 0, 0};
  std::vector<double> hpart(2 * std::max(nb, nbs));
  auto fft_w = [&](bool inv) -> fftmech_status {
    for (int w = 0; w < spec.nw; ++w) RC(fft_inplace(nx, ny, nz, true, inv, W[w], st));
    return FFTMECH_OK;
  };
  auto dot = [&](const cxd* a, const cxd* b, double& out) -> fftmech_status {
    CK(launch_var_dot(nU, a, b, part, st));
    CK(cudaMemcpyAsync(hpart.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out = 0.0;
    for (int i = 0; i < nb; ++i) out += hpart[i];
    return FFTMECH_OK;
  };
  auto precond = [&](const cxd* r, cxd* z) -> fftmech_status {
    for (int c = 0; c < dim; ++c) CK(launch_var_precond(g, r + (size_t)c * N, z + (size_t)c * N, st));
    return FFTMECH_OK;
  };
  // q = s D^H F[g C : (F^-1(sym D p) / N + Em - e I)]; p = NULL: the strain is Em - e I
  auto apply = [&](const cxd* p, cxd* q, const double* Em, const double* e, double s) -> fftmech_status {
    if (p) {
      CK(launch_varel_strain(g, spec, W, p, st));
      RC(fft_w(true));
    } else {
      for (int w = 0; w < spec.nw; ++w) CK(cudaMemsetAsync(W[w], 0, cb, st));
    }
    CK(launch_varel_stress(g, spec, W, phase, e, damage, kappa, lam, mu, Em, invN, st));
    RC(fft_w(false));
    CK(launch_varel_div(g, spec, W, s, q, st));
    return FFTMECH_OK;
  };
  RC(apply(nullptr, R, E, eig, -1.0));  // f_hat = -D^H F[g C : (E - e I)]
  CK(cudaMemsetAsync(X, 0, cu, st));
  RC(precond(R, Z));
  CK(cudaMemcpyAsync(P, Z, cu, cudaMemcpyDeviceToDevice, st));
  double rz = 0.0;
  RC(dot(R, Z, rz));
  const double rz0 = rz;
  const double tol2 = ctx->opts.tol * ctx->opts.tol;
  int it = 0;
  fftmech_status status = FFTMECH_OK;
  while (rz0 > 0.0 && rz > tol2 * rz0) {
    if (it >= ctx->opts.max_iter) {
      status = FFTMECH_ERR_NOT_CONVERGED;
      break;
    }
    RC(apply(P, Q, zero, nullptr, 1.0));
    double pq = 0.0;
    RC(dot(P, Q, pq));
    if (!(pq > 0.0) || !std::isfinite(pq)) {
      status = FFTMECH_ERR_NONFINITE;
      break;
    }
    const double alpha = rz / pq;
    CK(launch_var_axpy(nU, alpha, P, Q, X, R, st));
    RC(precond(R, Z));
    double rzn = 0.0;
    RC(dot(R, Z, rzn));
    ++it;
    CK(launch_var_dir(nU, rzn / rz, Z, P, st));
    rz = rzn;
  }
  // strain = E + F^-1(sym D u) / N, stress from it; their means
  CK(launch_varel_strain(g, spec, W, X, st));
  RC(fft_w(true));
  if (strain) {
    // the packed fields hold F^-1(sym D u); E is added per component below
    CK(launch_varel_real(g, spec, W, invN, strain, st));
  }
  double mean_eps[6] = {0, 0, 0, 0, 0, 0};
  for (int v = 0; v < spec.nv; ++v) mean_eps[v] = E[v];  // the fluctuation has zero mean
  CK(launch_varel_stress(g, spec, W, phase, eig, damage, kappa, lam, mu, E, invN, st));
  if (stress) CK(launch_varel_real(g, spec, W, 1.0, stress, st));
  double mean_sig[6] = {0, 0, 0, 0, 0, 0};
  for (int w = 0; w < spec.nw; ++w) {
    CK(launch_var_sum(N, W[w], part, st));
    CK(cudaMemcpyAsync(hpart.data(), part, 2 * nbs * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nbs; ++i) {
      a += hpart[2 * i];
      b += hpart[2 * i + 1];
    }
    mean_sig[2 * w] = a * invN;
    if (2 * w + 1 < spec.nv) mean_sig[2 * w + 1] = b * invN;
  }
  CK(cudaStreamSynchronize(st));
  std::memset(info, 0, sizeof(*info));
  info->status = status;
  info->iters = it;
  info->rel_res = rz0 > 0 ? std::sqrt(std::max(rz, 0.0) / rz0) : 0.0;
  info->true_rel_res = info->rel_res;
  for (int v = 0; v < spec.nv; ++v) {
    info->mean_stress[v] = mean_sig[v];
    info->mean_strain[v] = mean_eps[v];
  }
  // the strain output: add E to the fluctuation
  if (strain) {
    for (int v = 0; v < spec.nv; ++v)
      if (E[v] != 0.0) CK(launch_var_shift(N, E[v], strain + (size_t)v * N, st));
    CK(cudaStreamSynchronize(st));
  }
  return status;
}

// AT2 phase field with a chosen gradient operator (Eqs. crack, crack-fft with
// the symbol of Sec. 2.6): the history update of the library, then PCG on
// the spectrum of d. FP64, host-driven, one problem.
fftmech_status phasefield_operator_impl(fftmech_ctx* ctx, const uint8_t* phase, const double* strain,
                                        const double* eig, int op, bool literal, double* H, double* d,
                                        fftmech_solve_info* info) {
  using cxd = cx<double>;
  cudaStream_t st = ctx->stream;
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz, dim = ctx->dim;
  const long long N = ctx->N;
  const size_t cb = (size_t)N * sizeof(cxd);
  DevBuffers mem;
  cxd* P = mem.get<cxd>(cb);
  cxd* R = mem.get<cxd>(cb);
  cxd* X = mem.get<cxd>(cb);
  cxd* Z = mem.get<cxd>(cb);
  cxd* Q = mem.get<cxd>(cb);
  cxd* W = mem.get<cxd>(cb);
  double* Hd = mem.get<double>((size_t)N * sizeof(double));
  cxd* dx = mem.get<cxd>((size_t)nx * sizeof(cxd));
  cxd* dy = mem.get<cxd>((size_t)ny * sizeof(cxd));
  cxd* dz = mem.get<cxd>((size_t)nz * sizeof(cxd));
  const int nb = var_dot_blocks(N);
  double* part = mem.get<double>((size_t)2 * nb * sizeof(double));
  if (!mem.ok) return set_err(ctx, FFTMECH_ERR_OOM, "operator-variant buffers");
  const double h = ctx->h;
  const auto tx = grad_symbol(op, nx, h), ty = grad_symbol(op, ny, h), tz = grad_symbol(op, nz, h);
  CK(cudaMemcpyAsync(dx, tx.data(), nx * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dy, ty.data(), ny * sizeof(cxd), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dz, tz.data(), nz * sizeof(cxd), cudaMemcpyHostToDevice, st));
  const VarGrid g{nx, ny, nz, dim, N, dx, dy, dz};
  const double invN = 1.0 / (double)N;
  const double a = ctx->mat.Gc / (2.0 * ctx->mat.l0), b = ctx->mat.Gc * ctx->mat.l0 / 2.0;
  double lam[2], mu[2];
  lame(ctx->mat.E_pore, ctx->mat.nu_pore, lam[0], mu[0]);
  lame(ctx->mat.E_solid, ctx->mat.nu_solid, lam[1], mu[1]);
  // H = max(H, psi+(strain - e I)) (Eq. energy); m0 = a + <H>
  if (dim == 3)
    CK(launch3_history<double>(N, 1, phase, lam[0], lam[1], mu[0], mu[1], strain, eig, H, Hd, a, ctx->m0b,
                               ctx->partials, ctx->sc, st));
  else
    CK(launch_history<double>(N, 1, phase, lam[0], lam[1], mu[0], mu[1], strain, eig, H, Hd, a, ctx->m0b,
                              ctx->partials, ctx->sc, st));
  double m0 = 0.0;
  CK(cudaMemcpyAsync(&m0, ctx->m0b, sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<double> hpart(2 * nb);
  auto fft = [&](cxd* v, bool inv) -> fftmech_status { return fft_inplace(nx, ny, nz, true, inv, v, st); };
  auto dot = [&](const cxd* x, const cxd* y, double& out) -> fftmech_status {
    CK(launch_var_dot(N, x, y, part, st));
    CK(cudaMemcpyAsync(hpart.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out = 0.0;
    for (int i = 0; i < nb; ++i) out += hpart[i];
    return FFTMECH_OK;
  };
  // q = F[(a + H) F^-1(p) / N] + b |D|^2 p
  auto apply = [&](const cxd* p, cxd* q) -> fftmech_status {
    CK(cudaMemcpyAsync(W, p, cb, cudaMemcpyDeviceToDevice, st));
    RC(fft(W, true));
    CK(launch_varpf_react(N, Hd, a, invN, W, st));
    RC(fft(W, false));
    CK(launch_varpf_sum(g, b, literal ? 1 : 0, W, p, q, st));
    return FFTMECH_OK;
  };
  CK(launch_varpf_load(N, Hd, R, st));  // f_hat = F[H]
  RC(fft(R, false));
  CK(cudaStreamSynchronize(st));  // m0 on the host
  CK(cudaMemsetAsync(X, 0, cb, st));
  int it = 0;
  fftmech_status status = FFTMECH_OK;
  double rz = 0.0, rz0 = 0.0;
  if (literal) {
    // the printed Laplacian read literally is not symmetric: restarted
    // GMRES(m) with the Galerkin operator's diagonal as right
    // preconditioner, x = M y (Arnoldi by modified Gram-Schmidt, Givens
    // rotations; the host holds the small Hessenberg problem)
    constexpr int m = 40;
    DevBuffers vm;
    std::vector<cxd*> V(m + 1);
    for (auto& v : V) v = vm.get<cxd>(cb);
    cxd* Bv = vm.get<cxd>(cb);
    if (!vm.ok) return set_err(ctx, FFTMECH_ERR_OOM, "GMRES basis");
    CK(cudaMemcpyAsync(Bv, R, cb, cudaMemcpyDeviceToDevice, st));
    double bnorm2 = 0.0;
    RC(dot(Bv, Bv, bnorm2));
    const double bnorm = std::sqrt(bnorm2), tol = ctx->opts.tol;
    rz0 = bnorm2;
    rz = bnorm2;
    std::vector<double> Hm((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    auto Hij = [&](int i, int j) -> double& { return Hm[(size_t)i * m + j]; };
    while (bnorm > 0.0) {
      // R = b - A x
      if (it > 0) {
        RC(apply(X, Q));
        CK(cudaMemcpyAsync(R, Bv, cb, cudaMemcpyDeviceToDevice, st));
        CK(launch_var_scal(N, -1.0, Q, R, 1, st));
      }
      double beta2 = 0.0;
      RC(dot(R, R, beta2));
      const double beta = std::sqrt(beta2);
      rz = beta2;
      if (beta <= tol * bnorm) break;
      if (it >= ctx->opts.max_iter) {
        status = FFTMECH_ERR_NOT_CONVERGED;
        break;
      }
      CK(launch_var_scal(N, 1.0 / beta, R, V[0], 0, st));
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = beta;
      int k = 0;
      for (int j = 0; j < m && it < ctx->opts.max_iter; ++j) {
        CK(launch_varpf_precond(g, m0, b, V[j], Z, st));
        RC(apply(Z, V[j + 1]));
        for (int i = 0; i <= j; ++i) {
          RC(dot(V[i], V[j + 1], Hij(i, j)));
          CK(launch_var_scal(N, -Hij(i, j), V[i], V[j + 1], 1, st));
        }
        double hn2 = 0.0;
        RC(dot(V[j + 1], V[j + 1], hn2));
        const double hn = std::sqrt(hn2);
        if (hn > 0.0) CK(launch_var_scal(N, 1.0 / hn, V[j + 1], V[j + 1], 0, st));
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
          Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
          Hij(i, j) = t;
        }
        Hij(j + 1, j) = hn;
        const double den = std::hypot(Hij(j, j), hn);
        cs[j] = Hij(j, j) / den;
        sn[j] = hn / den;
        Hij(j, j) = den;
        Hij(j + 1, j) = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        k = j + 1;
        ++it;
        if (std::fabs(gv[j + 1]) <= tol * bnorm) break;
      }
      // x += M (sum y_i V_i), H y = g (upper triangular)
      for (int i = k - 1; i >= 0; --i) {
        double t = gv[i];
        for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
        y[i] = t / Hij(i, i);
      }
      CK(cudaMemsetAsync(P, 0, cb, st));
      for (int i = 0; i < k; ++i) CK(launch_var_scal(N, y[i], V[i], P, 1, st));
      CK(launch_varpf_precond(g, m0, b, P, Z, st));
      CK(launch_var_scal(N, 1.0, Z, X, 1, st));
    }
  }
  if (!literal) {
  CK(launch_varpf_precond(g, m0, b, R, Z, st));
  CK(cudaMemcpyAsync(P, Z, cb, cudaMemcpyDeviceToDevice, st));
  RC(dot(R, Z, rz));
  rz0 = rz;
  const double tol2 = ctx->opts.tol * ctx->opts.tol;
  while (rz0 > 0.0 && rz > tol2 * rz0) {
    if (it >= ctx->opts.max_iter) {
      status = FFTMECH_ERR_NOT_CONVERGED;
      break;
    }
    RC(apply(P, Q));
    double pq = 0.0;
    RC(dot(P, Q, pq));
    if (!(pq > 0.0) || !std::isfinite(pq)) {
      status = FFTMECH_ERR_NONFINITE;
      break;
    }
    const double alpha = rz / pq;
    CK(launch_var_axpy(N, alpha, P, Q, X, R, st));
    CK(launch_varpf_precond(g, m0, b, R, Z, st));
    double rzn = 0.0;
    RC(dot(R, Z, rzn));
    ++it;
    CK(launch_var_dir(N, rzn / rz, Z, P, st));
    rz = rzn;
  }
  }
  // d = F^-1(d_hat) / N; the total damage sum d = sum Re F^-1(d_hat) / N
  CK(cudaMemcpyAsync(W, X, cb, cudaMemcpyDeviceToDevice, st));
  RC(fft(W, true));
  if (d) CK(launch_var_real(g, W, nullptr, invN, d, nullptr, nullptr, st));
  CK(launch_var_sum(N, W, part, st));
  CK(cudaMemcpyAsync(hpart.data(), part, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double sd = 0.0;
  for (int i = 0; i < nb; ++i) sd += hpart[2 * i];
  std::memset(info, 0, sizeof(*info));
  info->status = status;
  info->iters = it;
  info->rel_res = rz0 > 0 ? std::sqrt(std::max(rz, 0.0) / rz0) : 0.0;
  info->true_rel_res = info->rel_res;
  info->total_damage = sd * invN;
  return status;
}

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
  if (!opts_ok(opts)) return FFTMECH_ERR_INVALID_ARG;
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
  for (cudaStream_t& s : ctx->side)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
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
    ctx->ds_rule = ctx->lshape.L_ds;
    choose_sten_shape(ctx->nx, ctx->ny, ctx->nz, grid->dim, ctx->nsm, batch, ctx->sshape);
  }
  if (!shp) return fail(FFTMECH_ERR_UNSUPPORTED_SIZE);
  ctx->shape.batch = batch;
  if (!three) {
    // reference-medium column pass: the widest strip (4, 2 or 1 columns and
    // their mirrors) that fits the shared memory and 512 threads
    const size_t es2 = fp64 ? 16 : 8;  // complex element
    for (int cw = 4; cw >= 1 && !ctx->ms_cw; cw /= 2) {
      const size_t sm = (size_t)ctx->ny * 2 * cw * es2 + (size_t)(ctx->ny + cw) * es2 +
                        (fp64 ? tw_smem_bytes<double>(ctx->ny) : tw_smem_bytes<float>(ctx->ny));
      const int thr = need_threads(ctx->py, 2 * cw);
      if (sm + 1024 <= ctx->optin && thr <= 512) {
        ctx->ms_cw = cw;
        ctx->ms_threads = std::min(512, std::max(128, round32(thr)));
      }
    }
  } else {
    // reference-medium z pass: the widest strip (4, 2 or 1 columns, six
    // slots of them) that fits the shared memory and 512 threads
    const int es2 = fp64 ? 16 : 8;
    for (int cw = 4; cw >= 1 && !ctx->ms3_cw; cw /= 2) {
      const size_t sm = zpass_ms_smem(ctx->nz, cw, es2,
                                      fp64 ? tw_smem_bytes<double>(ctx->nz) : tw_smem_bytes<float>(ctx->nz));
      const int thr = need_threads(ctx->pz, 6 * cw);
      if (sm + 1024 <= ctx->optin && thr <= 512) {
        ctx->ms3_cw = cw;
        ctx->ms3_threads = std::min(512, std::max(128, round32(thr)));
      }
    }
  }
  {
    double l1, m1s;
    lame(mat->E_solid, mat->nu_solid, l1, m1s);
    ctx->rho = l1 / m1s;
  }
  {
    // the rule-based shapes (a context never inherits another's tuning: its
    // reductions' block partitions, and so its last bits, depend only on
    // its own arguments and fftmech_autotune calls)
    const TuneChoice k = current_choice(ctx);
    snprintf(ctx->tune_desc, sizeof(ctx->tune_desc), "L_dir=%d L_upd=%d ty=%d zc=%d grid=%d cols=%d L_ds=%d",
             k.L_dir, k.L_upd, k.ty, k.zc, k.grid, k.cols, k.L_ds);
  }
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
    if (ctx->ms3_cw > 0) widest = std::max(widest, (size_t)zpass_ms_blocks(ctx->nx, ctx->ny, ctx->ms3_cw));
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
  ctx->rec_bytes = rec_total(ctx);
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) ok = false;
  };
  alloc(&ctx->q, nd * NB * es);
  alloc(&ctx->r, nd * NB * es);
  alloc(&ctx->p, nd * NB * es);
  if (!three) alloc(&ctx->pn, nd * NB * es);
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
  alloc(&ctx->ax, (size_t)(ctx->nx / 2 + 1) * 2 * es);
  alloc(&ctx->ay, (size_t)ctx->ny * 2 * es);
  if (three) {
    alloc(&ctx->az, (size_t)ctx->nz * 2 * es);
    alloc(&ctx->lamz, ctx->nz * es);
    alloc(&ctx->lamc3, (size_t)nxs_of(ctx->nx, 3) * es);
    alloc(&ctx->wcol3, (size_t)nxs_of(ctx->nx, 3) * es);
    alloc(&ctx->lamc1, (size_t)nxs_of(ctx->nx, 1) * es);
    alloc(&ctx->wcol1, (size_t)nxs_of(ctx->nx, 1) * es);
  }
  alloc((void**)&ctx->partials, slots * 8);
  if (!three) alloc((void**)&ctx->partials_col, (size_t)batch * ctx->nx * 8);
  alloc((void**)&ctx->m0b, (size_t)batch * 8);
  alloc((void**)&ctx->m1b, (size_t)batch * 8);
  alloc((void**)&ctx->mode, (size_t)batch * sizeof(int));
  alloc((void**)&ctx->sc, sizeof(SolverScalars) * batch);
  alloc((void**)&ctx->flags, sizeof(int) * LF_COUNT);
  alloc((void**)&ctx->rec, ctx->rec_bytes);
  if (!ok) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_flags, sizeof(int) * LF_COUNT) != cudaSuccess) return fail(FFTMECH_ERR_OOM);
  if (cudaMallocHost((void**)&ctx->h_rec, ctx->rec_bytes) != cudaSuccess) return fail(FFTMECH_ERR_OOM);
  std::memset(ctx->h_rec, 0, ctx->rec_bytes);
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
  for (GraphCache& c : ctx->gc)
    if (c.exec) cudaGraphExecDestroy(c.exec);
  void* bufs[] = {ctx->r, ctx->q, ctx->p, ctx->pn, ctx->S, ctx->g, ctx->uh, ctx->ul, ctx->phi, ctx->Hd,
                  ctx->cn, ctx->lamx, ctx->lamy, ctx->lamz, ctx->lamc3, ctx->lamc1, ctx->wcol3, ctx->wcol1,
                  ctx->ax, ctx->ay, ctx->az,
                  ctx->partials, ctx->partials_col, ctx->m0b, ctx->m1b, ctx->mode, ctx->sc, ctx->flags, ctx->rec};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < ST_COUNT; ++i)
    if (ctx->stage[i].dev) cudaFree(ctx->stage[i].dev);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  if (ctx->h_rec) cudaFreeHost(ctx->h_rec);
  for (auto& pe : ctx->pending) { ctx->ev_free.push_back(pe.a); ctx->ev_free.push_back(pe.b); }
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  for (cudaStream_t s : ctx->side)
    if (s) cudaStreamDestroy(s);
  free_plan(ctx->px);
  free_plan(ctx->py);
  free_plan(ctx->pz);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return FFTMECH_OK;
}

fftmech_status fftmech_set_solver_opts(fftmech_ctx* ctx, const fftmech_solver_opts* opts) {
  if (!ctx || !opts) return FFTMECH_ERR_INVALID_ARG;
  if (!opts_ok(opts)) return FFTMECH_ERR_INVALID_ARG;
  ctx->opts = *opts;
  if (ctx->opts.check_every <= 0) ctx->opts.check_every = 16;
  return FFTMECH_OK;
}

int fftmech_batch_size(const fftmech_ctx* ctx) { return ctx ? ctx->B : 0; }

fftmech_status fftmech_set_launch_shapes(fftmech_ctx* ctx, const char* shapes) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!shapes) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "shapes must not be NULL");
  TuneChoice c = current_choice(ctx);
  const char* s = shapes;
  for (;;) {
    while (*s == ' ') ++s;
    if (!*s || *s == '(') break;  // the end, or a "(cached)" note
    char key[16] = {0};
    int val = 0, used = 0;
    if (std::sscanf(s, "%15[A-Za-z_]=%d%n", key, &val, &used) != 2 || used <= 0)
      return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "shapes: expected key=value");
    const std::string k(key);
    if (k == "L_dir") c.L_dir = val;
    else if (k == "L_upd") c.L_upd = val;
    else if (k == "ty") c.ty = val;
    else if (k == "zc") c.zc = val;
    else if (k == "grid") c.grid = val;
    else if (k == "cols") c.cols = val;
    else if (k == "L_ds") c.L_ds = val;
    else return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "shapes: unknown key");
    s += used;
  }
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  if (c.L_ds < 0 || !(fp64 ? choice_ok<double>(ctx, c) : choice_ok<float>(ctx, c)))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "shapes: not a valid launch shape for this grid");
  if (fp64) apply_choice<double>(ctx, c);
  else apply_choice<float>(ctx, c);
  snprintf(ctx->tune_desc, sizeof(ctx->tune_desc), "L_dir=%d L_upd=%d ty=%d zc=%d grid=%d cols=%d L_ds=%d", c.L_dir,
           c.L_upd, c.ty, c.zc, c.grid, c.cols, c.L_ds);
  return FFTMECH_OK;
}

fftmech_status fftmech_autotune(fftmech_ctx* ctx, int iterations, double* before_us, double* after_us,
                                const char** choice) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (iterations < 0) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "iterations must be >= 0");
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  if (iterations > 0) {
    // a choice tuned earlier in the process for the same device, grid,
    // batch and precision is applied without timing again
    TuneEntry c;
    bool have = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(tune_key(ctx));
      if (it != g_tune.end()) {
        c = it->second;
        have = true;
      }
    }
    if (have && (fp64 ? choice_ok<double>(ctx, c.choice) : choice_ok<float>(ctx, c.choice))) {
      if (fp64) apply_choice<double>(ctx, c.choice);
      else apply_choice<float>(ctx, c.choice);
      if (before_us) *before_us = c.before_us;
      if (after_us) *after_us = c.after_us;
      const TuneChoice& k = c.choice;
      snprintf(ctx->tune_desc, sizeof(ctx->tune_desc),
               "L_dir=%d L_upd=%d ty=%d zc=%d grid=%d cols=%d L_ds=%d (cached)", k.L_dir, k.L_upd, k.ty, k.zc, k.grid,
               k.cols, k.L_ds);
    } else {
      rc = fp64 ? autotune_impl<double>(ctx, iterations, before_us, after_us)
                : autotune_impl<float>(ctx, iterations, before_us, after_us);
    }
  }
  if (choice) *choice = ctx->tune_desc;
  return rc;
}

fftmech_status fftmech_adjoint_eigenstrain(fftmech_ctx* ctx, const uint8_t* phase, const void* e_field, int steps,
                                           const double* ramp, const double eps_mac[6], int objective,
                                           int checkpoint_every, double* grad, double* J,
                                           fftmech_solve_info* info_last) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !e_field || !ramp || !grad || !J || steps < 1 || checkpoint_every < 1)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument or bad count");
  if (objective != FFTMECH_OBJ_ENERGY && objective != FFTMECH_OBJ_DAMAGE)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "objective %d", objective);
  if (ctx->B != 1) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "the adjoint takes one problem per context");
  for (const void* p : {(const void*)phase, e_field, (const void*)grad})
    if (!is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "the adjoint takes device pointers");
  double E[6] = {0, 0, 0, 0, 0, 0};
  if (eps_mac)
    for (int i = 0; i < nvoigt(ctx); ++i) E[i] = eps_mac[i];
  const int k = std::min(checkpoint_every, steps);
  return ctx->prec == FFTMECH_FP64
             ? adjoint_impl<double>(ctx, phase, (const double*)e_field, steps, ramp, E, objective, k, grad, J, info_last)
             : adjoint_impl<float>(ctx, phase, (const float*)e_field, steps, ramp, E, objective, k, grad, J, info_last);
}

fftmech_status fftmech_homogenise_operator(fftmech_ctx* ctx, const uint8_t* phase, int gradient,
                                          const double grad_c_mac[3], double* phi, double* grad_c,
                                          fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !grad_c_mac || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (gradient < FFTMECH_GRAD_FORWARD || gradient > FFTMECH_GRAD_FOURIER)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "gradient operator %d", gradient);
  if (ctx->B != 1) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "one problem per context");
  for (const void* p : {(const void*)phase, (const void*)phi, (const void*)grad_c})
    if (p && !is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "device pointers only");
  if (gradient == FFTMECH_GRAD_FOURIER && (ctx->nx % 2 == 0 || (ctx->dim >= 2 && ctx->ny % 2 == 0) ||
                                           (ctx->dim == 3 && ctx->nz % 2 == 0)))
    return set_err(ctx, FFTMECH_ERR_UNSUPPORTED_SIZE, "the Fourier gradient needs odd grid sizes");
  double G[3] = {0, 0, 0};
  for (int k = 0; k < ctx->dim; ++k) G[k] = grad_c_mac[k];
  return homogenise_operator_impl(ctx, phase, gradient, G, phi, grad_c, info);
}

fftmech_status fftmech_equilibrium_operator(fftmech_ctx* ctx, const uint8_t* phase, const double* eig,
                                            const double* damage, const double eps_mac[6], int gradient,
                                            double* strain, double* stress, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !eps_mac || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (gradient < FFTMECH_GRAD_FORWARD || gradient > FFTMECH_GRAD_FOURIER)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "gradient operator %d", gradient);
  if (ctx->B != 1) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "one problem per context");
  for (const void* p : {(const void*)phase, (const void*)eig, (const void*)damage, (const void*)strain,
                        (const void*)stress})
    if (p && !is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "device pointers only");
  if (gradient == FFTMECH_GRAD_FOURIER && (ctx->nx % 2 == 0 || (ctx->dim >= 2 && ctx->ny % 2 == 0) ||
                                           (ctx->dim == 3 && ctx->nz % 2 == 0)))
    return set_err(ctx, FFTMECH_ERR_UNSUPPORTED_SIZE, "the Fourier gradient needs odd grid sizes");
  double E[6] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < nvoigt(ctx); ++k) E[k] = eps_mac[k];
  return equilibrium_operator_impl(ctx, phase, eig, damage, E, gradient, strain, stress, info);
}

fftmech_status fftmech_phasefield_operator(fftmech_ctx* ctx, const uint8_t* phase, const double* strain,
                                           const double* eig, int gradient, double* H, double* d,
                                           fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !strain || !H || !d || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  const bool literal = (gradient & FFTMECH_PF_LITERAL) != 0;
  gradient &= ~FFTMECH_PF_LITERAL;
  if (gradient < FFTMECH_GRAD_FORWARD || gradient > FFTMECH_GRAD_FOURIER)
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "gradient operator %d", gradient);
  if (ctx->B != 1) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "one problem per context");
  for (const void* p : {(const void*)phase, (const void*)strain, (const void*)eig, (const void*)H, (const void*)d})
    if (p && !is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "device pointers only");
  if (gradient == FFTMECH_GRAD_FOURIER && (ctx->nx % 2 == 0 || (ctx->dim >= 2 && ctx->ny % 2 == 0) ||
                                           (ctx->dim == 3 && ctx->nz % 2 == 0)))
    return set_err(ctx, FFTMECH_ERR_UNSUPPORTED_SIZE, "the Fourier gradient needs odd grid sizes");
  return phasefield_operator_impl(ctx, phase, strain, eig, gradient, literal, H, d, info);
}

fftmech_status fftmech_problem_offset(const fftmech_ctx* ctx, int problem, int components, long long* offset) {
  if (!ctx || !offset || problem < 0 || problem >= ctx->B || components < 1) return FFTMECH_ERR_INVALID_ARG;
  *offset = (long long)problem * components * ctx->N;
  return FFTMECH_OK;
}

fftmech_status fftmech_graph_stats(const fftmech_ctx* ctx, long long* builds, long long* launches,
                                   long long* kernels, int* disabled, const char** reason) {
  if (!ctx) return FFTMECH_ERR_INVALID_ARG;
  if (builds) *builds = ctx->graph_builds;
  if (launches) *launches = ctx->graph_launches;
  if (kernels) *kernels = ctx->graph_kernels;
  if (disabled) *disabled = ctx->graph_off ? 1 : 0;
  if (reason) *reason = ctx->graph_err;
  return FFTMECH_OK;
}

fftmech_status fftmech_equilibrium_solve(fftmech_ctx* ctx, const uint8_t* phase, const void* eig,
                                         const double* damage, const double eps_mac[6], double* u,
                                         void* strain, void* stress, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!phase || !eps_mac || !u || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(fftmech_solve_info) * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  void *dphase, *deig, *ddmg, *du, *dstrain, *dstress;
  RC(stage_in(ctx, ST_PHASE, phase, N, true, &dphase));
  RC(stage_in(ctx, ST_EIG, eig, N * es, true, &deig));
  RC(stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &ddmg));
  RC(stage_in(ctx, ST_U, u, (size_t)ctx->dim * N * 8, true, &du));
  RC(stage_in(ctx, ST_STRAIN, strain, nv * N * es, false, &dstrain));
  RC(stage_in(ctx, ST_STRESS, stress, nv * N * es, false, &dstress));
  double E[6];
  for (int k = 0; k < 6; ++k) E[k] = k < (int)nv ? eps_mac[k] : 0.0;
  std::vector<unsigned char> key;
  for (const void* p : {dphase, deig, ddmg, du, dstrain, dstress}) key_add(key, p);
  key_add(key, E);
  key_add(key, ctx->opts);
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  RC(run_op(ctx, OP_EQ, key, [&](Emit& em) -> fftmech_status {
    if (fp64)
      RC(enqueue_equilibrium<double>(em, (const uint8_t*)dphase, (const double*)deig, (const double*)ddmg, E,
                                     (double*)du, (double*)dstrain, (double*)dstress));
    else
      RC(enqueue_equilibrium<float>(em, (const uint8_t*)dphase, (const float*)deig, (const double*)ddmg, E,
                                    (double*)du, (float*)dstrain, (float*)dstress));
    return rec_publish(em);
  }));
  ctx->last = LastOp();
  ctx->last.valid = 1;
  ctx->last.ran[SK_EQ] = 1;
  ctx->last.lc = ctx->pending_lc;
  RC(stage_out(ctx, u, du, (size_t)ctx->dim * N * 8));
  RC(stage_out(ctx, strain, dstrain, nv * N * es));
  RC(stage_out(ctx, stress, dstress, nv * N * es));
  RC(finish_sync(ctx));
  count_graph_kernels(ctx);
  return collect(ctx, SK_EQ, info, 1);
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
  if (mode == FFTMECH_DIFF_TRANSIENT && !(dt > 0))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt must be > 0 for TRANSIENT");
  std::memset(info, 0, sizeof(fftmech_solve_info) * ctx->B);
  const size_t N = (size_t)ctx->N * ctx->B;
  void *dphase, *dc, *dmask = nullptr;
  RC(stage_in(ctx, ST_PHASE, phase, N, true, &dphase));
  RC(stage_in(ctx, ST_C, c, N * 8, mode == FFTMECH_DIFF_TRANSIENT, &dc));
  if (mode == FFTMECH_DIFF_TRANSIENT) RC(stage_in(ctx, ST_MASK, dirichlet_mask, N, true, &dmask));
  double G[3] = {0, 0, 0};
  if (grad_c_mac)
    for (int k = 0; k < 3; ++k) G[k] = grad_c_mac[k];
  std::vector<unsigned char> key;
  for (const void* p : {dphase, dc, dmask}) key_add(key, p);
  key_add(key, mode);
  key_add(key, G);
  key_add(key, c_macro);
  key_add(key, dt);
  key_add(key, dirichlet_value);
  key_add(key, ctx->opts);
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  RC(run_op(ctx, OP_DIFF, key, [&](Emit& em) -> fftmech_status {
    if (fp64)
      RC(enqueue_diffusion<double>(em, (const uint8_t*)dphase, mode, G, c_macro, dt, (const uint8_t*)dmask,
                                   dirichlet_value, (double*)dc));
    else
      RC(enqueue_diffusion<float>(em, (const uint8_t*)dphase, mode, G, c_macro, dt, (const uint8_t*)dmask,
                                  dirichlet_value, (double*)dc));
    return rec_publish(em);
  }));
  ctx->last = LastOp();
  ctx->last.valid = 1;
  ctx->last.ran[SK_DIFF] = 1;
  ctx->last.diff_mode = mode;
  ctx->last.c_macro = c_macro;
  ctx->last.lc = ctx->pending_lc;
  RC(stage_out(ctx, c, dc, N * 8));
  RC(finish_sync(ctx));
  count_graph_kernels(ctx);
  return collect(ctx, SK_DIFF, info, 1);
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
  RC(stage_in(ctx, ST_STRAIN, strain, nv * N * es, true, &dstrain));
  RC(stage_in(ctx, ST_EIG, eig, N * es, true, &deig));
  RC(stage_in(ctx, ST_PHASE, phase, N, true, &dphase));
  RC(stage_in(ctx, ST_H, H, N * es, true, &dH));
  RC(stage_in(ctx, ST_DAMAGE, damage, N * 8, true, &dd));
  std::vector<unsigned char> key;
  for (const void* p : {dstrain, deig, dphase, dH, dd}) key_add(key, p);
  key_add(key, ctx->opts);
  const bool fp64 = ctx->prec == FFTMECH_FP64;
  RC(run_op(ctx, OP_PF, key, [&](Emit& em) -> fftmech_status {
    if (fp64)
      RC(enqueue_phasefield<double>(em, (const double*)dstrain, (const double*)deig, (const uint8_t*)dphase,
                                    (double*)dH, (double*)dd));
    else
      RC(enqueue_phasefield<float>(em, (const float*)dstrain, (const float*)deig, (const uint8_t*)dphase,
                                   (float*)dH, (double*)dd));
    return rec_publish(em);
  }));
  ctx->last = LastOp();
  ctx->last.valid = 1;
  ctx->last.ran[SK_PF] = 1;
  ctx->last.lc = ctx->pending_lc;
  RC(stage_out(ctx, H, dH, N * es));
  RC(stage_out(ctx, damage, dd, N * 8));
  RC(finish_sync(ctx));
  count_graph_kernels(ctx);
  return collect(ctx, SK_PF, info, 1);
}

fftmech_status fftmech_staggered_step(fftmech_ctx* ctx, fftmech_state* state,
                                      const fftmech_step_params* prm, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  RC(check_step_args(ctx, state, prm));
  std::memset(info, 0, sizeof(fftmech_solve_info) * 3 * ctx->B);
  StepPtrs d;
  bool all_device = false;
  RC(stage_step(ctx, state, prm, d, all_device));
  RC(step_enqueue(ctx, d, prm));
  const size_t N = (size_t)ctx->N * ctx->B, es = esize(ctx), nv = nvoigt(ctx);
  RC(stage_out(ctx, state->c, d.c, N * 8));
  RC(stage_out(ctx, state->c_ppt, d.cppt, N * es));
  RC(stage_out(ctx, state->eig, d.eig, N * es));
  RC(stage_out(ctx, state->u, d.u, (size_t)ctx->dim * N * 8));
  RC(stage_out(ctx, state->strain, d.strain, nv * N * es));
  RC(stage_out(ctx, state->stress, d.stress, nv * N * es));
  RC(stage_out(ctx, state->H, d.H, N * es));
  RC(stage_out(ctx, state->damage, d.d, N * 8));
  RC(finish_sync(ctx));
  return step_collect(ctx, info);
}

fftmech_status fftmech_staggered_step_async(fftmech_ctx* ctx, const fftmech_state* state,
                                            const fftmech_step_params* prm) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  RC(check_step_args(ctx, state, prm));
  StepPtrs d;
  bool all_device = false;
  // every pointer must be device memory: nothing is staged, copied or allocated
  const void* ptrs[] = {state->phase, state->c, state->c_ppt, state->eig, state->u, state->strain, state->stress,
                        state->H, state->damage,
                        prm->diffusion_mode == FFTMECH_DIFF_TRANSIENT ? (const void*)prm->dirichlet_mask : nullptr,
                        prm->eig_mode == FFTMECH_EIG_PRESCRIBED ? prm->eig_field : nullptr};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "host pointer in an asynchronous step");
  RC(stage_step(ctx, state, prm, d, all_device));
  return step_enqueue(ctx, d, prm);
}

fftmech_status fftmech_step_info(fftmech_ctx* ctx, fftmech_solve_info* info) {
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  if (!ctx->last.valid || !ctx->last.ran[SK_EQ])
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "no staggered step has been enqueued");
  RC(finish_sync(ctx));
  return step_collect(ctx, info);
}

fftmech_status fftmech_bar_create(fftmech_bar** out, fftmech_ctx* ctx, double length, double dt, double flux_in,
                                  const double* c0) {
  if (!out) return FFTMECH_ERR_INVALID_ARG;
  *out = nullptr;
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  const int M = ctx->B;
  if (!(length > 0) || !(dt > 0) || !std::isfinite(flux_in))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "bar length and dt must be > 0");
  const double dX = length / M;
  const double dmax = std::max(ctx->mat.D_pore, ctx->mat.D_solid);
  if (dt > dX * dX / (2.0 * dmax))
    return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "dt %g above the explicit bound dX^2 / (2 D_max) = %g", dt,
                   dX * dX / (2.0 * dmax));
  fftmech_bar* b = new (std::nothrow) fftmech_bar();
  if (!b) return FFTMECH_ERR_OOM;
  b->ctx = ctx;
  const size_t n = (size_t)(M + 1) + 4 * (size_t)M;
  if (cudaMalloc(&b->mem, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return set_err(ctx, FFTMECH_ERR_OOM, "bar buffers");
  }
  b->d.M = M;
  b->d.dX = dX;
  b->d.dt = dt;
  b->d.flux_in = flux_in;
  b->d.c = b->mem;
  b->d.cbar = b->mem + M + 1;
  b->d.G = b->d.cbar + M;
  std::vector<double> h(n, 0.0);
  if (c0) std::memcpy(h.data(), c0, sizeof(double) * (M + 1));
  if (cudaMemcpy(b->mem, h.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->mem);
    delete b;
    return set_err(ctx, FFTMECH_ERR_CUDA, "bar upload");
  }
  *out = b;
  return FFTMECH_OK;
}

fftmech_status fftmech_bar_destroy(fftmech_bar* bar) {
  if (!bar) return FFTMECH_ERR_INVALID_ARG;
  if (bar->ctx) cudaStreamSynchronize(bar->ctx->stream);
  cudaFree(bar->mem);
  delete bar;
  return FFTMECH_OK;
}

fftmech_status fftmech_bar_step(fftmech_bar* bar, const fftmech_state* state, const fftmech_step_params* params,
                                fftmech_solve_info* info) {
  if (!bar) return FFTMECH_ERR_INVALID_ARG;
  fftmech_ctx* ctx = bar->ctx;
  fftmech_status rc = check_ctx(ctx);
  if (rc != FFTMECH_OK) return rc;
  if (!params || !info) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "null argument");
  fftmech_step_params prm = *params;
  prm.diffusion_mode = FFTMECH_DIFF_HOMOGENISE;
  prm.c_macro = 0.0;
  for (double& g : prm.grad_c_mac) g = 0.0;
  prm.c_macro_each = bar->d.cbar;
  prm.grad_c_mac_each = bar->d.G;
  RC(check_step_args(ctx, state, &prm));
  const void* ptrs[] = {state->phase, state->c, state->c_ppt, state->eig, state->u, state->strain, state->stress,
                        state->H, state->damage,
                        prm.eig_mode == FFTMECH_EIG_PRESCRIBED ? prm.eig_field : nullptr};
  for (const void* p : ptrs)
    if (p && !is_device_ptr(p)) return set_err(ctx, FFTMECH_ERR_INVALID_ARG, "the bar takes device pointers");
  StepPtrs d;
  bool all_device = false;
  RC(stage_step(ctx, state, &prm, d, all_device));
  RC(step_enqueue(ctx, d, &prm, &bar->d));
  RC(finish_sync(ctx));
  return step_collect(ctx, info);
}

fftmech_status fftmech_bar_read(const fftmech_bar* bar, double* c_host) {
  if (!bar || !c_host) return FFTMECH_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(bar->ctx->stream) != cudaSuccess ||
      cudaMemcpy(c_host, bar->d.c, sizeof(double) * (bar->d.M + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FFTMECH_ERR_CUDA;
  }
  return FFTMECH_OK;
}

fftmech_status fftmech_bar_write(fftmech_bar* bar, const double* c_host) {
  if (!bar || !c_host) return FFTMECH_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(bar->ctx->stream) != cudaSuccess ||
      cudaMemcpy(bar->d.c, c_host, sizeof(double) * (bar->d.M + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return FFTMECH_ERR_CUDA;
  }
  return FFTMECH_OK;
}

fftmech_status fftmech_group_create(fftmech_group** out, fftmech_ctx* const* ctxs, int n, void* stream) {
  if (!out || !ctxs || n < 1) return FFTMECH_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return FFTMECH_ERR_INVALID_ARG;
    if (ctxs[i]->device != ctxs[0]->device) return FFTMECH_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->stream == ctxs[i]->stream) return FFTMECH_ERR_INVALID_ARG;
  }
  fftmech_group* g = new (std::nothrow) fftmech_group();
  if (!g) return FFTMECH_ERR_OOM;
  g->ctxs.assign(ctxs, ctxs + n);
  g->lc.resize(n);
  auto fail = [&](fftmech_status s) {
    fftmech_group_destroy(g);
    return s;
  };
  if (cudaSetDevice(ctxs[0]->device) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
    g->own_stream = true;
  }
  for (int i = 0; i < n; ++i)
    if (ctxs[i]->stream == g->stream) return fail(FFTMECH_ERR_INVALID_ARG);
  if (cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
  g->join.assign(n, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) != cudaSuccess) return fail(FFTMECH_ERR_CUDA);
  *out = g;
  return FFTMECH_OK;
}

fftmech_status fftmech_group_destroy(fftmech_group* g) {
  if (!g) return FFTMECH_ERR_INVALID_ARG;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->fork) cudaEventDestroy(g->fork);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return FFTMECH_OK;
}

const char* fftmech_group_last_error(const fftmech_group* g) { return g ? g->err : ""; }

fftmech_status fftmech_group_step(fftmech_group* g, const fftmech_state* const* states,
                                  const fftmech_step_params* const* params, fftmech_solve_info* const* infos) {
  if (!g || !states || !params || !infos) return FFTMECH_ERR_INVALID_ARG;
  g->err[0] = 0;
  const int n = (int)g->ctxs.size();
  if (cudaSetDevice(g->ctxs[0]->device) != cudaSuccess) return FFTMECH_ERR_CUDA;
  std::vector<StepPtrs> d(n);
  std::vector<unsigned char> key;
  for (int i = 0; i < n; ++i) {
    fftmech_ctx* ctx = g->ctxs[i];
    ctx->err[0] = 0;
    if (!states[i] || !params[i] || !infos[i]) return FFTMECH_ERR_INVALID_ARG;
    fftmech_status rc = check_step_args(ctx, states[i], params[i]);
    if (rc != FFTMECH_OK) {
      snprintf(g->err, sizeof(g->err), "problem group %d: %s", i, ctx->err);
      return rc;
    }
    bool all_device = false;
    RC(stage_step(ctx, states[i], params[i], d[i], all_device));
    if (!all_device) {
      snprintf(g->err, sizeof(g->err), "problem group %d: host pointer (a group runs on device memory)", i);
      return FFTMECH_ERR_INVALID_ARG;
    }
    key_add(key, ctx);
    key_add(key, d[i]);
    key_add(key, *params[i]);
    key_add(key, ctx->opts);
  }
  if (!g->exec || key != g->key) {
    // capture: fork every context's stream from the group stream, emit its
    // step there (conditional nodes included), join back
    fftmech_ctx* ctx = g->ctxs[0];  // for CK's messages
    if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      snprintf(g->err, sizeof(g->err), "cudaStreamBeginCapture failed");
      return FFTMECH_ERR_CUDA;
    }
    fftmech_status rc = FFTMECH_OK;
    std::vector<LaunchCount> lc(n);
    if (cudaEventRecord(g->fork, g->stream) != cudaSuccess) rc = FFTMECH_ERR_CUDA;
    for (int i = 0; i < n && rc == FFTMECH_OK; ++i) {
      fftmech_ctx* c = g->ctxs[i];
      if (cudaStreamWaitEvent(c->stream, g->fork, 0) != cudaSuccess) { rc = FFTMECH_ERR_CUDA; break; }
      Emit em = eager_emit(c);
      em.graph = true;
      em.lc = &lc[i];
      cudaStreamCaptureStatus cs;
      if (cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &em.g, nullptr, nullptr, nullptr) != cudaSuccess) {
        rc = FFTMECH_ERR_CUDA;
        break;
      }
      const bool fp64 = c->prec == FFTMECH_FP64;
      rc = fp64 ? enqueue_step<double>(em, d[i], params[i]) : enqueue_step<float>(em, d[i], params[i]);
      if (rc == FFTMECH_OK) rc = rec_publish(em);
      if (rc != FFTMECH_OK) snprintf(g->err, sizeof(g->err), "problem group %d: %s", i, c->err);
      if (rc == FFTMECH_OK && (cudaEventRecord(g->join[i], c->stream) != cudaSuccess ||
                               cudaStreamWaitEvent(g->stream, g->join[i], 0) != cudaSuccess))
        rc = FFTMECH_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    if (rc == FFTMECH_OK && e != cudaSuccess) rc = FFTMECH_ERR_CUDA;
    if (rc == FFTMECH_OK && g->exec) {
      cudaGraphExecUpdateResultInfo ri;
      if (cudaGraphExecUpdate(g->exec, graph, &ri) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
      }
    }
    if (rc == FFTMECH_OK && !g->exec && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      g->exec = nullptr;
      rc = FFTMECH_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != FFTMECH_OK) {
      cudaGetLastError();
      if (!g->err[0]) snprintf(g->err, sizeof(g->err), "building the group graph failed");
      return rc;
    }
    g->key = key;
    g->lc = lc;
    g->builds += 1;
    (void)ctx;
  }
  const cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
  if (e == cudaSuccess) g->launches += 1;
  const cudaError_t es = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess || es != cudaSuccess) {
    cudaGetLastError();
    snprintf(g->err, sizeof(g->err), "group graph: %s", cudaGetErrorString(e != cudaSuccess ? e : es));
    return FFTMECH_ERR_CUDA;
  }
  fftmech_status worst = FFTMECH_OK;
  for (int i = 0; i < n; ++i) {
    fftmech_ctx* ctx = g->ctxs[i];
    const fftmech_step_params* prm = params[i];
    ctx->last = LastOp();
    ctx->last.valid = 1;
    ctx->last.ran[SK_DIFF] = prm->diffusion_mode != FFTMECH_DIFF_NONE;
    ctx->last.ran[SK_EQ] = ctx->last.ran[SK_PF] = 1;
    ctx->last.diff_mode = prm->diffusion_mode;
    ctx->last.c_macro = prm->c_macro;
    ctx->last.lc = &g->lc[i];
    const long long before = ctx->graph_kernels;
    const fftmech_status s = step_collect(ctx, infos[i]);
    g->kernels += ctx->graph_kernels - before;
    if (s != FFTMECH_OK && worst == FFTMECH_OK) worst = s;
  }
  return worst;
}

fftmech_status fftmech_group_stats(const fftmech_group* g, long long* builds, long long* launches,
                                   long long* kernels) {
  if (!g) return FFTMECH_ERR_INVALID_ARG;
  if (builds) *builds = g->builds;
  if (launches) *launches = g->launches;
  if (kernels) *kernels = g->kernels;
  return FFTMECH_OK;
}

fftmech_status fftmech_staggered_step_many(fftmech_ctx* const* ctxs, int n, fftmech_state* const* states,
                                           const fftmech_step_params* const* params,
                                           fftmech_solve_info* const* infos) {
  if (!ctxs || !states || !params || !infos || n < 0) return FFTMECH_ERR_INVALID_ARG;
  if (n == 0) return FFTMECH_OK;
  fftmech_group* g = nullptr;
  fftmech_status rc = fftmech_group_create(&g, ctxs, n, nullptr);
  if (rc != FFTMECH_OK) return rc;
  rc = fftmech_group_step(g, states, params, infos);
  fftmech_group_destroy(g);
  return rc;
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
  if (!n || !data || ndim < 1 || ndim > 3) return FFTMECH_ERR_INVALID_ARG;
  if (precision != FFTMECH_FP64 && precision != FFTMECH_MIXED) return FFTMECH_ERR_INVALID_ARG;
  if (!is_device_ptr(data)) return FFTMECH_ERR_INVALID_ARG;
  const int nx = n[0], ny = ndim >= 2 ? n[1] : 1, nz = ndim == 3 ? n[2] : 1;
  cudaStream_t st = (cudaStream_t)stream;
  fftmech_status rc = fft_inplace(nx, ny, nz, precision == FFTMECH_FP64, inverse != 0, data, st);
  if (rc != FFTMECH_OK) return rc;
  return cudaStreamSynchronize(st) == cudaSuccess ? FFTMECH_OK : FFTMECH_ERR_CUDA;
}

}  // extern "C"
