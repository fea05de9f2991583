// Internal declarations shared by the kernel translation units and the C ABI
// layer: operator / vector parameter blocks, device-side solver scalars and
// the host launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "fftmech_dev.cuh"

namespace fftmech {

// Launch mode of the calling host thread for the PCG kernels: nonzero =
// programmatic dependent launches (each kernel's launch and constant
// prologue overlap the end of the previous kernel on the stream), 0 = plain
// stream order. The solver sets it for the duration of a solve (DepLaunchScope).
extern thread_local int tl_dependent_launch;

struct DepLaunchScope {
  int saved;
  explicit DepLaunchScope(int on) : saved(tl_dependent_launch) { tl_dependent_launch = on; }
  ~DepLaunchScope() { tl_dependent_launch = saved; }
};

// Launch a kernel that calls grid_dep_sync() first in every block (only
// such kernels may be launched this way), with the programmatic
// stream-serialisation attribute when the thread's mode asks for it.
template <typename... KA, typename... A>
cudaError_t launch_dep(void (*kernel)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = tl_dependent_launch ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Opt a kernel into the device's full dynamic shared memory. The attribute
// is per device, so the flag that skips repeated calls is one bit per device
// (devices 0..63; a device beyond that is configured on every call).
// Launches then pass their own, smaller, sizes.
struct SmemOptIn {
  std::atomic<unsigned long long> done{0};
};
template <typename K>
static cudaError_t opt_in_smem(K kernel, size_t bytes, SmemOptIn& flag) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (flag.done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in limit
  if ((long long)bytes > (long long)dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e == cudaSuccess && bit) flag.done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Scalars of one PCG run, resident in device memory. The last block of a
// reduction kernel updates them; every iteration kernel reads `done` first.
struct SolverScalars {
  double rz;       // <r, M^-1 r> of the current residual
  double rz0;      // <f, M^-1 f> of the right-hand side (the normaliser)
  double pq;       // <p, K p>
  double alpha, beta;
  double tol2;     // tol^2
  double rz_true;  // <r, M^-1 r> right after the last true-residual replacement
  int iter, max_iter, done, status;
  unsigned int cnt[4];  // last-block counters: 0 direction, 1 column pass, 2 stats
  // deferred reductions (2D): <r, M^-1 r> of the last column pass, taken by
  // the direction kernel's blocks and committed to rz by block 0 of the
  // kernel after them (commit_pending_rz); col_true: that column pass
  // followed a reliable update
  double rz_next;
  int col_true, pad_i;
  // float copies for the float kernels (no FP64 instruction in their hot
  // path): alpha = alpha_h + alpha_l, beta rounded
  float alpha_h, alpha_l, beta_f, pad_f;
  // reliable updates (MIXED): <r, M^-1 r> right after the last residual
  // replacement (or the first residual); reliable: replacements enabled;
  // nrestart: restarts taken after a recursive convergence; nreplace:
  // replacement iterations scheduled
  double rz_rep;
  int reliable, nrestart, nreplace;
  // deferred reductions (2D): rz_next holds the residual norm still to be
  // committed to rz (with iter += 1)
  int rz_pending;
  // the FP64 true residual of this stopped problem is in rz_true (set by the
  // gate after its true-residual pass; cleared by a restart), so later
  // rounds of a batch do not recompute it
  int checked;
};

// Loop control of the device-driven PCG. The kernels that decide whether a
// loop continues store their decision in `flags` (device memory, read by
// the host when the solve runs without a graph) and, when the solve runs as
// a CUDA graph, also set the conditional node's value. Exactly one thread
// of a launch sets a given condition (concurrent cudaGraphSetConditional
// calls on one handle are not allowed).
// LF_LOOP: run another ordinary iteration; LF_REPLACE: the next iteration
// replaces a residual (reliable update); LF_GATE: some problem has stopped
// and its FP64 true residual has not been checked yet (the gate's
// true-residual passes run); LF_OUTER: the solve goes on (set before the
// first iteration, cleared by the restart gate); LF_RESTART: some problem
// restarts from its true residual.
// LF_ROUNDS (not a condition) counts the outer rounds of a solve; the gate
// ends a solve whose rounds exceed max_iter + 64.
enum LoopFlag { LF_LOOP = 0, LF_REPLACE = 1, LF_OUTER = 2, LF_RESTART = 3, LF_GATE = 4, LF_ROUNDS = 5, LF_COUNT = 6 };
struct LoopCtl {
  int* flags;                      // LF_COUNT ints (NULL: no loop control in this launch)
  unsigned long long h[LF_COUNT];  // cudaGraphConditionalHandle per flag (graph mode)
  unsigned int have;               // bit k: h[k] is valid in the graph being run
  int direct;                      // 1: one problem; the direction kernel sets LF_LOOP, LF_REPLACE, LF_GATE
};

// Column-pass modes: ITER (one PCG iteration: beta, convergence), NORM
// (<f, M^-1 f> -> rz0, no store), INIT (first residual), PLAIN (bare column
// FFT), TRUE (iteration right after a true-residual replacement),
// TRUENORM (<r, M^-1 r> of a true residual -> rz_true, no store), RESTART
// (true residual after a recursive convergence: restart with beta = 0).
enum ColMode {
  COL_ITER = 0, COL_NORM = 1, COL_INIT = 2, COL_PLAIN = 3, COL_TRUE = 4, COL_TRUENORM = 5,
  COL_RESTART = 6
};
// Flag or-ed into COL_ITER (2D): store one partial per block and leave the
// finalisation to the next direction kernel (deferred reduction).
constexpr int COL_DEFER = 16;


// Material / operator description for the row kernels (2D: nz = 1).
// Vector (D = d, elasticity): K u = grad+^T [g C_omega : sym grad+ u];
//   residual r = -grad+^T [g C_omega : (E + sym grad+ u - e I)].
// Scalar (D = 1): K u = c0(x) u + grad+^T [kap_omega grad+ u];
//   residual r = P (src - c0 u - grad+^T [kap_omega (grad+ u + G)]),
//   c0 = c0c + c0f(x), src = src_scale * (srcd or srct), P zeroes masked voxels.
template <typename T>
struct Op {
  int nx, ny, nz;
  double h;
  const uint8_t* phase;
  // elasticity
  const T* g;  // degradation per voxel (NULL = 1)
  double lam[2], mu[2];  // by phase: [0] pore, [1] solid
  const T* eig;  // isotropic eigenstrain (NULL = 0)
  double E[6];   // macro strain: 2D xx, yy, xy; 3D xx, yy, zz, yz, xz, xy
  // scalar problems
  double kap[2];
  double c0c;
  const T* c0f;
  const uint8_t* mask;
  double G[3];
  // per-problem macro gradient (3 per problem) and macro concentration of a
  // batch (device; NULL: G and the call's c_macro for every problem)
  const double* Gp;
  const double* cmp;
  const double* srcd;
  const T* srct;
  double src_scale;
  // the constants above rounded to T by the host (the float kernels use
  // these, so they convert nothing per thread): 1/h, lam, mu, kap, c0c
  T ih_t, lam_t[2], mu_t[2], kap_t[2], c0c_t;
  // elasticity: a prescribed stress field tau (Voigt, nv x N; NULL = 0)
  // subtracted from the stress in the residual, r = -grad+^T [sigma - tau]:
  // the right-hand side grad+^T tau of the equilibrium adjoint
  const T* pre;
};

// Macro concentration gradient component k of problem b.
template <typename T>
__device__ __forceinline__ double macro_grad(const Op<T>& op, int b, int k) {
  return op.Gp ? op.Gp[3 * b + k] : op.G[k];
}

// The iterate: double in FP64; in MIXED an unevaluated float pair
// u = uh + ul (double-float arithmetic: Knuth's TwoSum, Dekker's product
// split via FMA) so the hot loop needs no FP64 instruction.
template <typename T>
struct Vec2 {
  double* u;      // iterate, D x N (FP64 path)
  float* uh;      // MIXED: high part, D x N
  float* ul;      // MIXED: low part, D x N
  T* r;           // residual, D x N
  const T* p_in;  // previous direction (update kernel: the current one)
  T* p_out;       // new direction
  T* p_copy;      // update kernel: where it also stores the current direction (NULL: nowhere)
  cx<T>* S;       // spectral rows, N complex (components packed re / im)
  T* q;           // K p (split iteration), D x N
  double* partials;
  SolverScalars* sc;  // one per problem of the batch
  // deferred reductions (2D): the column pass's partials and their count
  // per problem (0: the last column pass finalised itself), the stencil's
  // partial count per problem (0: the stencil finalised alpha itself), and
  // whether rz_next holds the residual norm to commit
  const double* pcol;
  int ncol, nsten;
  int* mode;    // per problem: 0 normal, 1 reliable update, 2 restart (NULL = all 0)
  LoopCtl ctl;  // loop decisions of the direction kernel
};

// Problems of a uniform batch sit back to back: problem b's scalar fields at
// b N, its d-component fields at b d N, its spectrum at b N, its scalars at
// sc + b; launches put the problem index in blockIdx.y.
template <typename T, int D>
__device__ __forceinline__ void problem_views(Op<T>& op, Vec2<T>& v, int b, size_t N) {
  const size_t o1 = (size_t)b * N, oD = (size_t)b * D * N;
  op.phase += o1;
  if (op.g) op.g += o1;
  if (op.eig) op.eig += o1;
  if (op.c0f) op.c0f += o1;
  if (op.mask) op.mask += o1;
  if (op.srcd) op.srcd += o1;
  if (op.srct) op.srct += o1;
  if (op.pre) op.pre += (size_t)b * (D == 3 ? 6 : 3) * N;
  if (v.u) v.u += oD;
  if (v.uh) v.uh += oD;
  if (v.ul) v.ul += oD;
  v.r += oD;
  if (v.p_in) v.p_in += oD;
  if (v.p_out) v.p_out += oD;
  v.S += o1;
  v.sc += b;
}

// Fourier multiplier 1 / (m0 + m1 lambda(k)), lambda = lamx[kx] + lamy[ky]
// (the symbol of grad+^T grad+); 0 where the denominator is 0 (k = 0 when
// m0 = 0), scaled by 1/N to fold the inverse transform's normalisation.
// 3D line passes: lambda = lamc[spectral column] + lamj[line set] +
// laml[line], Parseval weight wcol[spectral column].
template <typename T>
struct Spec {
  const T* lamx;
  const T* lamy;
  double m0, m1;
  double invN;
  const double* m0b;  // per-problem m0 (NULL = m0 for all)
  const double* m1b;  // per-problem m1 (NULL = m1 for all)
  const T* lamc;
  const T* lamj;
  const T* laml;
  const T* wcol;
  T m0_t, m1_t, invN_t;  // m0, m1, invN rounded to T by the host
  // reference-medium preconditioner (elasticity; NULL = Laplace): D h per
  // mode along x (columns 0 .. nx / 2), y and z (3D), and lambda0 / mu0
  const cx<T>* ax;
  const cx<T>* ay;
  const cx<T>* az;
  T rho_t;
};

// Launch shapes chosen by the host.
struct Shape2 {
  int batch;  // problems of a uniform batch (grid.y of the solver kernels)
  int rows_update, threads_update;
  int rows_dir, threads_dir;
  int rows_res, threads_res;
  int cols, threads_col;
  int threads_plain;
};

// 3D launch shapes: FP64 residual bricks of ry lines x zc planes, and
// strips of cw spectral columns for the y and z passes.
struct Shape3 {
  int batch;
  int nx, ny, nz;
  long long sst;  // complex numbers per problem in the spectral buffer
  int ry_res, zc_res, thr_res;
  int cw_y, thr_y;
  int cw_z, thr_z;
};

// Split iteration (lines.cuh, stencil.cuh): x-line kernels take L whole
// lines per block; stencil kernels TX x TY tiles (x TZ planes in 3D).
struct LineShape {
  int batch;
  long long sst;  // complex numbers per problem in the spectral buffer
  int L_dir, thr_dir;
  int L_upd, thr_upd;
  int L_ds, thr_ds;  // fused direction-stencil kernel (2D; L_ds = 0: not available)
};
struct StenShape {
  int batch;
  int tx, ty, zc, threads;
  int grid;  // blocks per problem (they loop over the tiles)
};

// Blocks per problem of the 2D stencil (warp strips of 30 columns and s.ty
// rows, 8 warps a block, at most s.grid blocks).
inline int sten2_blocks(int nx, int ny, const StenShape& s) {
  const int items = ((nx + 29) / 30) * ((ny + s.ty - 1) / s.ty);
  const int blocks = (items + 7) / 8;
  return s.grid > 0 ? std::min(s.grid, blocks) : blocks;
}
// Blocks per problem of the 3D stencil (bricks of 30 columns, s.ty rows and
// s.zc planes, 8 warps a block, at most s.grid blocks).
inline int sten3_blocks(int nx, int ny, int nz, const StenShape& s) {
  const long long items = (long long)((nx + 29) / 30) * ((ny + s.ty - 1) / s.ty) * ((nz + s.zc - 1) / s.zc);
  const long long blocks = (items + 7) / 8;
  return (int)(s.grid > 0 ? std::min<long long>(s.grid, blocks) : blocks);
}


// ---------------------------------------------------------------- launchers
// Row kernels take the radix family of the x transform (FX), column kernels
// that of the y transform (FY); see RadixFamily.
template <typename T, int D, int FX>
cudaError_t launch_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                            const Shape2& sh, int zero_u, int filter, cudaStream_t st);
template <typename T, int FY, int NY, int CWC>
cudaError_t launch_colpass(int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp,
                           const Shape2& sh, int mode, int inverse, double* partials,
                           SolverScalars* sc, int* pmode, cudaStream_t st);
template <typename T, int FX>
cudaError_t launch_rowfft(int nx, int ny, cx<T>* S, const FftPlanDev<T>& px, int inverse,
                          const Shape2& sh, cudaStream_t st);

// Line lengths with compile-time FFT kernels (float): the benchmark grids
// (3^4 .. 3^7 and 2^7 .. 2^10).
#define FFTMECH_FIXED_SWITCH(n, CALL) \
  switch (n) {                        \
    case 81: return CALL(81);         \
    case 243: return CALL(243);       \
    case 729: return CALL(729);       \
    case 2187: return CALL(2187);     \
    case 128: return CALL(128);       \
    case 256: return CALL(256);       \
    case 512: return CALL(512);       \
    case 1024: return CALL(1024);     \
    default: break;                   \
  }

#define FFTMECH_FAMILY_SWITCH(fam, CALL)      \
  switch (fam) {                              \
    case FAM_9: return CALL(FAM_9);           \
    case FAM_93: return CALL(FAM_93);         \
    case FAM_842: return CALL(FAM_842);       \
    default: return CALL(FAM_ALL);            \
  }

template <typename T, int D>
inline cudaError_t launch_residual_f(int fx, const Op<T>& op, const Vec2<T>& v,
                                     const FftPlanDev<T>& px, const Shape2& sh, int zero_u,
                                     int filter, cudaStream_t st) {
#define FFTMECH_C(F) launch_residual<T, D, F>(op, v, px, sh, zero_u, filter, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}
template <typename T>
inline cudaError_t launch_colpass_f(int fy, int nx, int ny, cx<T>* S, const FftPlanDev<T>& py,
                                    const Spec<T>& sp, const Shape2& sh, int mode, int inverse,
                                    double* partials, SolverScalars* sc, int* pmode,
                                    cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    // compile-time column plans for the benchmark lengths and strip widths
#define FFTMECH_CW(NY)                                                                                  \
  (sh.cols == 8   ? launch_colpass<T, FAM_ALL, NY, 8>(nx, ny, S, py, sp, sh, mode, inverse, partials, sc, pmode, st) \
   : sh.cols == 4 ? launch_colpass<T, FAM_ALL, NY, 4>(nx, ny, S, py, sp, sh, mode, inverse, partials, sc, pmode, st) \
                  : launch_colpass<T, FAM_ALL, NY, 2>(nx, ny, S, py, sp, sh, mode, inverse, partials, sc, pmode, st))
    if (sh.cols == 2 || sh.cols == 4 || sh.cols == 8) {
      FFTMECH_FIXED_SWITCH(ny, FFTMECH_CW)
    }
#undef FFTMECH_CW
  }
#define FFTMECH_C(F) launch_colpass<T, F, 0, 0>(nx, ny, S, py, sp, sh, mode, inverse, partials, sc, pmode, st)
  FFTMECH_FAMILY_SWITCH(fy, FFTMECH_C)
#undef FFTMECH_C
}
// Column pass with the reference-medium preconditioner (colpass_ms.cu): one
// block per strip of CW columns kx <= nx / 2 and their mirrors nx - kx.
inline int colpass_ms_blocks(int nx, int CW) { return (nx / 2 + 1 + CW - 1) / CW; }
// z pass with the reference-medium preconditioner (zpass_ms.cu, 3D): one
// block per pair of line sets (ky, ny - ky) and strip of CW columns
// kx <= nx / 2; shared memory for nz rows of six CW-column slots.
int zpass_ms_blocks(int nx, int ny, int CW);
size_t zpass_ms_smem(int nz, int CW, int es_complex, size_t tw);
template <typename T>
cudaError_t launch3_zpass_ms_f(int fz, cx<T>* S, long long sst, int nx, int ny, int nz, int nxs,
                               const FftPlanDev<T>& pz, const Spec<T>& sp, int CW, int threads, int batch, int mode,
                               double* partials, SolverScalars* sc, int* pmode, cudaStream_t st);
template <typename T>
cudaError_t launch_colpass_ms_f(int fy, int nx, int ny, cx<T>* S, const FftPlanDev<T>& py, const Spec<T>& sp,
                                int CW, int threads, int batch, int mode, double* partials, SolverScalars* sc,
                                int* pmode, cudaStream_t st);

template <typename T>
inline cudaError_t launch_rowfft_f(int fx, int nx, int ny, cx<T>* S, const FftPlanDev<T>& px,
                                   int inverse, const Shape2& sh, cudaStream_t st) {
#define FFTMECH_C(F) launch_rowfft<T, F>(nx, ny, S, px, inverse, sh, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}

// 3D launchers (kernels3d.cuh); axis 1 = y pass, 2 = z pass; stage 0 / 1 / 2
// = forward FFT / multiplier pass / inverse FFT.
template <typename T, int D, int FX>
cudaError_t launch3_residual(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const Shape3& sh,
                             int zero_u, int filter, cudaStream_t st);
template <typename T, int FL, int NL, int CWC>
cudaError_t launch3_lines(cx<T>* S, const Shape3& sh, int D, int axis, int stage, const FftPlanDev<T>& pl,
                          const Spec<T>& sp, int mode, double* partials, SolverScalars* sc, int* pmode,
                          cudaStream_t st);

template <typename T, int D>
inline cudaError_t launch3_residual_f(int fx, const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                                      const Shape3& sh, int zero_u, int filter, cudaStream_t st) {
#define FFTMECH_C(F) launch3_residual<T, D, F>(op, v, px, sh, zero_u, filter, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}
template <typename T>
inline cudaError_t launch3_lines_f(int fl, cx<T>* S, const Shape3& sh, int D, int axis, int stage,
                                   const FftPlanDev<T>& pl, const Spec<T>& sp, int mode, double* partials,
                                   SolverScalars* sc, int* pmode, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    const int cw = axis == 1 ? sh.cw_y : sh.cw_z;
    if (cw == 16) {
#define FFTMECH_C(NL) launch3_lines<T, FAM_ALL, NL, 16>(S, sh, D, axis, stage, pl, sp, mode, partials, sc, pmode, st)
      FFTMECH_FIXED_SWITCH(pl.n, FFTMECH_C)
#undef FFTMECH_C
    }
  }
#define FFTMECH_C(F) launch3_lines<T, F, 0, 0>(S, sh, D, axis, stage, pl, sp, mode, partials, sc, pmode, st)
  FFTMECH_FAMILY_SWITCH(fl, FFTMECH_C)
#undef FFTMECH_C
}

// Split iteration launchers; x-line kernels take the radix family of the x
// transform, DIM the grid dimension.
template <typename T, int D, int FX, int DIM, int NX>
cudaError_t launch_xdir(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                        cudaStream_t st);
template <typename T, int D, int FX, int DIM, int NX>
cudaError_t launch_xupd(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                        cudaStream_t st);

template <typename T, int D, int FX, int NX>
cudaError_t launch_xds(const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px, const LineShape& ls,
                       cudaStream_t st);

template <typename T, int D>
cudaError_t launch_sten2(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st);
template <typename T, int D>
cudaError_t launch_sten3(const Op<T>& op, const Vec2<T>& v, const StenShape& ss, cudaStream_t st);

template <typename T, int D, int DIM>
inline cudaError_t launch_xdir_f(int fx, const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                                 const LineShape& ls, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
#define FFTMECH_C(NX) launch_xdir<T, D, FAM_ALL, DIM, NX>(op, v, px, ls, st)
    FFTMECH_FIXED_SWITCH(px.n, FFTMECH_C)
#undef FFTMECH_C
  }
#define FFTMECH_C(F) launch_xdir<T, D, F, DIM, 0>(op, v, px, ls, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}
template <typename T, int D>
inline cudaError_t launch_xds_f(int fx, const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                                const LineShape& ls, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
#define FFTMECH_C(NX) launch_xds<T, D, FAM_ALL, NX>(op, v, px, ls, st)
    FFTMECH_FIXED_SWITCH(px.n, FFTMECH_C)
#undef FFTMECH_C
  }
#define FFTMECH_C(F) launch_xds<T, D, F, 0>(op, v, px, ls, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}
template <typename T, int D, int DIM>
inline cudaError_t launch_xupd_f(int fx, const Op<T>& op, const Vec2<T>& v, const FftPlanDev<T>& px,
                                 const LineShape& ls, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
#define FFTMECH_C(NX) launch_xupd<T, D, FAM_ALL, DIM, NX>(op, v, px, ls, st)
    FFTMECH_FIXED_SWITCH(px.n, FFTMECH_C)
#undef FFTMECH_C
  }
#define FFTMECH_C(F) launch_xupd<T, D, F, DIM, 0>(op, v, px, ls, st)
  FFTMECH_FAMILY_SWITCH(fx, FFTMECH_C)
#undef FFTMECH_C
}

// Post-processing and pointwise kernels (2D); `batch` problems (grid.y).
template <typename T>
cudaError_t launch_el_output(const Op<T>& op, int batch, const double* u, T* strain, T* stress,
                             double* partials, double* results, SolverScalars* sc, cudaStream_t st);
template <typename T>
cudaError_t launch_diff_stats(const Op<T>& op, int batch, const double* phi, double hdiff,
                              double c_macro, double* partials, double* results, SolverScalars* sc,
                              cudaStream_t st);
cudaError_t launch_diff_write_c(int nx, int ny, int batch, const uint8_t* phase, const double* phi,
                                double hdiff, double G0, double G1, const double* Gp, const double* beta_dev,
                                double* c, cudaStream_t st);
template <typename T>
cudaError_t launch_history(long long N, int batch, const uint8_t* phase, double lam0, double lam1,
                           double mu0, double mu1, const T* strain, const T* eig, T* H, double* Hd,
                           double a, double* m0b, double* partials, SolverScalars* sc,
                           cudaStream_t st);
cudaError_t launch_pf_stats(long long N, int batch, const uint8_t* phase, const double* d,
                            double* partials, double* results, SolverScalars* sc, double Dp,
                            double Ds, double ih2, double* m1b, cudaStream_t st);
template <typename T>
cudaError_t launch_degradation(long long N, const double* d, double kappa, T* g, cudaStream_t st);
template <typename T>
cudaError_t launch_precipitate(long long N, const uint8_t* phase, const double* c, double S,
                               double M, T* c_ppt, T* eig, cudaStream_t st);
template <typename T>
cudaError_t launch_scale_copy(long long N, const T* src, double scale, T* dst, cudaStream_t st);
cudaError_t launch_set_masked(long long N, const uint8_t* mask, double value, double* c,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_to_real(long long N, const double* src, T* dst, cudaStream_t st);
cudaError_t launch_df_split(long long n, const double* u, float* uh, float* ul, cudaStream_t st);
// Deferred column-pass finalisation (see k_col_finalize), one block per problem.
cudaError_t launch_col_finalize(const double* pcol, int ncol, SolverScalars* sc, int batch, double invN, int fp32,
                                cudaStream_t st);
cudaError_t launch_df_merge(long long n, const float* uh, const float* ul, double* u, cudaStream_t st);

// Homogenised diffusion with a chosen gradient operator (variants.cu).
struct VarGrid {
  int nx, ny, nz, dim;
  long long N;
  const cx<double>* dx;  // gradient symbol along x (nx values), y, z
  const cx<double>* dy;
  const cx<double>* dz;
};
int var_dot_blocks(long long n);
// Elasticity with a chosen gradient operator: Voigt components (tensor
// shears) as index pairs (a, b), packed two per complex field.
struct VarElSpec {
  int nv, nw;
  int a[6], b[6];
};
VarElSpec var_el_spec(int dim);
cudaError_t launch_var_shift(long long n, double c, double* x, cudaStream_t st);
// Phase field with a chosen gradient operator.
cudaError_t launch_varpf_load(long long n, const double* f, cx<double>* W, cudaStream_t st);
cudaError_t launch_varpf_react(long long n, const double* H, double a, double invN, cx<double>* W, cudaStream_t st);
cudaError_t launch_varpf_sum(const VarGrid& g, double b, int literal, const cx<double>* W, const cx<double>* P,
                             cx<double>* Q, cudaStream_t st);
cudaError_t launch_var_scal(long long n, double c, const cx<double>* x, cx<double>* y, int add, cudaStream_t st);
cudaError_t launch_varpf_precond(const VarGrid& g, double m0, double b, const cx<double>* r, cx<double>* z,
                                 cudaStream_t st);
cudaError_t launch_varel_strain(const VarGrid& g, const VarElSpec& sp, cx<double>* const* W, const cx<double>* U,
                                cudaStream_t st);
cudaError_t launch_varel_stress(const VarGrid& g, const VarElSpec& sp, cx<double>* const* W, const uint8_t* phase,
                                const double* eig, const double* damage, double kappa, const double lam[2],
                                const double mu[2], const double E[6], double invN, cudaStream_t st);
cudaError_t launch_varel_div(const VarGrid& g, const VarElSpec& sp, cx<double>* const* W, double s,
                             cx<double>* Q, cudaStream_t st);
cudaError_t launch_varel_real(const VarGrid& g, const VarElSpec& sp, cx<double>* const* W, double scale,
                              double* out, cudaStream_t st);
cudaError_t launch_var_grad(const VarGrid& g, const cx<double>* P, cx<double>* W1, cx<double>* W2, cudaStream_t st);
cudaError_t launch_var_flux(const VarGrid& g, const uint8_t* phase, double kp, double ks, const double G[3],
                            double invN, cx<double>* W1, cx<double>* W2, cudaStream_t st);
cudaError_t launch_var_div(const VarGrid& g, const cx<double>* Z1, const cx<double>* Z2, double s, cx<double>* Q,
                           cudaStream_t st);
cudaError_t launch_var_dot(long long n, const cx<double>* a, const cx<double>* b, double* partials,
                           cudaStream_t st);
cudaError_t launch_var_sum(long long n, const cx<double>* w, double* partials, cudaStream_t st);
cudaError_t launch_var_axpy(long long n, double alpha, const cx<double>* p, const cx<double>* q, cx<double>* x,
                            cx<double>* r, cudaStream_t st);
cudaError_t launch_var_precond(const VarGrid& g, const cx<double>* r, cx<double>* z, cudaStream_t st);
cudaError_t launch_var_dir(long long n, double beta, const cx<double>* z, cx<double>* p, cudaStream_t st);
cudaError_t launch_var_real(const VarGrid& g, const cx<double>* W1, const cx<double>* W2, double scale, double* gx,
                            double* gy, double* gz, cudaStream_t st);

// Macroscale bar (bar.cu).
cudaError_t launch_bar_inputs(int M, double dX, const double* c, double* cbar, double* G, cudaStream_t st);
cudaError_t launch_bar_update(int M, double dX, double dt, double flux_in, double* c, const double* res, int stride,
                              cudaStream_t st);

// Reverse sweep of the staggered solve (adjoint.cu).
cudaError_t launch_fill(long long N, double v, double* p, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_m0b(long long N, const T* H, double a, double* m0b, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_history(int dim, long long N, const uint8_t* phase, double lam0, double lam1, double mu0,
                               double mu1, const T* strain, const T* efield, double scale, const T* Hprev,
                               const double* d, const double* lam_pf, const double* lam_inv, double* dJ_dH, T* tau,
                               double* dJde, double* ddirect, int energy_last, const double* dprev, double kappa,
                               double vol, cudaStream_t st);
template <typename T>
cudaError_t launch_adj_eqpost(int dim, int nx, int ny, int nz, const uint8_t* phase, double lam0, double lam1,
                              double mu0, double mu1, const T* strain, const T* efield, double scale,
                              const double* dprev, double kappa, const double* mu, const double* mu_inv, double h,
                              const double* dJde, const double* ddirect, double* dJdd, double* grad,
                              cudaStream_t st);
// x *= 2^k chosen so that max |x| lands in [target / 2, target); scale[0] =
// 2^k, scale[1] = 2^-k on the device (m: one 8-byte scratch slot).
template <typename X>
cudaError_t launch_adj_normalise(long long n, X* x, unsigned long long* m, double target, double* scale,
                                 cudaStream_t st);

// Control kernels of the device-driven PCG (control.cu).
cudaError_t launch_sc_init(SolverScalars* sc, int batch, double tol2, int max_iter, int reliable, cudaStream_t st);
cudaError_t launch_zero_rhs(double* u, float* uh, float* ul, long long n, SolverScalars* sc, int batch, int has_mask,
                            cudaStream_t st);
cudaError_t launch_loopctl(const SolverScalars* sc, const int* mode, int batch, const LoopCtl& ctl,
                           cudaStream_t st);
cudaError_t launch_gate(SolverScalars* sc, int* mode, int batch, const LoopCtl& ctl, int max_rounds, cudaStream_t st);
cudaError_t launch_sync_flags(const LoopCtl& ctl, cudaStream_t st);
cudaError_t launch_clear_modes(int* mode, int batch, cudaStream_t st);
cudaError_t launch_set_flag(const LoopCtl& ctl, int k, int value, cudaStream_t st);
cudaError_t launch_stamp(unsigned long long* slot, cudaStream_t st);

// 3D post-processing (post3d.cu): results[b * 13 + k] (6 stress sums, 6
// strain sums, energy) and results[b * 6 + k] (beta_pore, beta_solid, 3 mean
// fluxes, porosity).
template <typename T>
cudaError_t launch3_el_output(const Op<T>& op, int batch, const double* u, T* strain, T* stress, double* partials,
                              double* results, SolverScalars* sc, cudaStream_t st);
template <typename T>
cudaError_t launch3_diff_stats(const Op<T>& op, int batch, const double* phi, double hdiff, double c_macro,
                               double* partials, double* results, SolverScalars* sc, cudaStream_t st);
cudaError_t launch3_diff_write_c(int nx, int ny, int nz, int batch, const uint8_t* phase, const double* phi,
                                 double hdiff, const double G[3], const double* Gp, const double* beta_dev,
                                 double* c, cudaStream_t st);
template <typename T>
cudaError_t launch3_history(long long N, int batch, const uint8_t* phase, double lam0, double lam1, double mu0,
                            double mu1, const T* strain, const T* eig, T* H, double* Hd, double a, double* m0b,
                            double* partials, SolverScalars* sc, cudaStream_t st);

// Shared-memory layouts of the row kernels for tiles of R rows of nx
// (byte offsets, each region 16-byte aligned), used by host and device.
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// residual (FP64 stencil): [P: max(D (R+2) doubles, 2 R T) per column]
// [SG: 3 (R+1) doubles per column]
template <typename T, int D>
inline size_t smem_residual(int nx, int R) {
  const size_t a = (size_t)D * (R + 2) * sizeof(double), b = (size_t)2 * R * sizeof(T);
  return align16((a > b ? a : b) * nx) + (size_t)3 * (R + 1) * nx * sizeof(double);
}
// 3D spectral rows: D = 3 stores the packed (x, y) components (nx complex)
// and the z component's half spectrum (nx/2 + 1); D = 1 the half spectrum.
__host__ __device__ inline int nxs_of(int nx, int D) { return (D == 3 ? nx : 0) + nx / 2 + 1; }

// 3D FP64 residual bricks: [P: two planes x D (R+2) lines, double] [SP:
// in-plane stress or flux, NP (R+1) lines] [SZ: z-differenced components,
// two planes x NZ (R+1) lines] [F: NF R complex lines of T] [MG: g or c0
// field, R+1 lines of T] [PH: phase bytes, R+1 lines] [MK: mask bytes, R
// lines]
struct Row3Layout {
  size_t P, SP, SZ, F, MG, PH, MK, total;
  __host__ __device__ Row3Layout(int nx, int R, int cs, int ts, int D) {
    const size_t np = D == 3 ? 3 : 2, nzc = D == 3 ? 3 : 1, nf = D == 3 ? 2 : 1;
    const size_t L = (size_t)nx;
    P = 0;
    SP = P + align16((size_t)2 * D * (R + 2) * L * cs);
    SZ = SP + align16(np * (R + 1) * L * cs);
    F = SZ + align16(2 * nzc * (R + 1) * L * cs);
    MG = F + align16(nf * R * L * 2 * ts);
    PH = MG + align16((size_t)(R + 1) * L * ts);
    MK = PH + align16((size_t)(R + 1) * L);
    total = MK + align16((size_t)R * L);
  }
};

// Fused direction-stencil kernel (2D, L own rows per block): [F: max(L + 2
// complex rows, NS (L + 1) rows of stress components)] [PO: D (L + 2) rows
// of the direction] [MG: (L + 1) rows of the material field] [PH: (L + 1)
// rows of phase bytes] [MK: (L + 2) rows of mask bytes], after the
// twiddles.
template <typename T, int D>
struct DsLayout {
  static constexpr int NS = D == 2 ? 3 : 2;  // stress (xx, yy, xy) or flux (x, y) components
  size_t F, PO, MG, PH, MK, total;
  __host__ __device__ DsLayout(int nx, int L) {
    const size_t rows_f = (size_t)(L + 2) * nx * sizeof(cx<T>);
    const size_t rows_s = (size_t)NS * (L + 1) * nx * sizeof(T);
    F = 0;
    PO = align16(rows_f > rows_s ? rows_f : rows_s);
    MG = PO + align16((size_t)D * (L + 2) * nx * sizeof(T));
    PH = MG + align16((size_t)(L + 1) * nx * sizeof(T));
    MK = PH + align16((size_t)(L + 1) * nx);
    total = MK + align16((size_t)(L + 2) * nx);
  }
};

// Split-iteration shared memory (bytes, including the staged twiddles).
template <typename T>
inline size_t xdir_smem(int nx, int L, int D, int dim) {
  const int nf = (dim == 3 && D == 3) ? 2 : 1;
  return tw_smem_bytes<T>(nx) + align16((size_t)nf * L * nx * sizeof(cx<T>)) +
         align16((size_t)D * L * nx * sizeof(T)) + (size_t)L * nx;  // + Dirichlet mask bytes
}
template <typename T>
inline size_t xupd_smem(int nx, int L, int D, int dim) {
  const int nf = (dim == 3 && D == 3) ? 2 : 1;
  return tw_smem_bytes<T>(nx) + (size_t)nf * L * nx * sizeof(cx<T>);
}



}  // namespace fftmech
