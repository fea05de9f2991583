/*
 * fftmech: FFT-Galerkin corrosion-fracture hot path on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library libfftmech.so. It computes, on voxel grids of a
 * two-phase porous microstructure, the steps of one staggered load step of
 * Pundir, Kammer & Angst, "An FFT-based framework for predicting
 * corrosion-driven damage in fractal porous media" (arXiv 2305.13081):
 * ionic diffusion (Sec. 2.1), precipitation and eigenstrain (Sec. 2.2),
 * mechanical equilibrium (Sec. 2.3) and the phase-field damage (Sec. 2.4), in
 * the order of Algorithm 1 (Sec. 2.5).
 *
 * Discretisation (Sec. 2.1, 2.6, App. A). Fields live on the voxels of a
 * periodic grid with spacing h. Gradients use the forward-difference symbol
 * D_a(k) = (exp(i 2 pi k_a / n_a) - 1) / h of Sec. 2.6; the compatibility
 * projections G and GG of App. A (Eq. g-42) are applied as
 * "backward-difference divergence -> Fourier multiplier 1/|D|^2 ->
 * forward-difference gradient", which is the same operator, so each
 * Galerkin system is solved as a preconditioned CG on the potential
 * (displacement u, concentration fluctuation phi, damage d) whose iterates map
 * one to one onto the paper's gradient-space CG iterates.
 *
 * Conventions shared by every entry point
 * - Layout: structure of arrays, C order, x fastest: a scalar field is
 *   n[1]*n[0] (2D) or n[2]*n[1]*n[0] (3D) elements; a d-component field is d
 *   such blocks back to back. Tensor fields use Voigt order xx, yy, xy (2D)
 *   or xx, yy, zz, yz, xz, xy (3D) with TENSOR shear components (not
 *   engineering strains).
 * - Phase indicator omega (uint8 per voxel): 1 = solid, 0 = pore (Sec. 2.1).
 * - Element types: "iterate" fields (u, c, damage) are always double.
 *   "Field" arrays (eigenstrain, strain, stress, history H, c_ppt) are
 *   double for FFTMECH_FP64 and float for FFTMECH_MIXED.
 * - Pointers may be device pointers (cudaMalloc, torch CUDA tensors) or host
 *   pointers (pageable or pinned); host buffers are staged through
 *   library-owned device memory on the context's stream.
 * - Ownership: the caller owns every field buffer; the library owns only its
 *   workspace (allocated in fftmech_create, freed in fftmech_destroy).
 * - Synchronisation: every compute entry point enqueues its work on the
 *   context's CUDA stream and returns after that work has completed, with
 *   `info` filled in on the host; fftmech_staggered_step_async returns at
 *   once and its reports are read with fftmech_step_info.
 * - Allocation: with device pointers no call after fftmech_create
 *   allocates device memory. Host pointers are staged through device
 *   buffers that the library allocates on first use (kept until
 *   fftmech_destroy).
 * - Errors: argument errors return before any work is enqueued. Solver
 *   outcomes (converged, not converged, non-finite) are returned as the
 *   status and also stored in info->status. A CUDA failure returns
 *   FFTMECH_ERR_CUDA; fftmech_last_error() gives the message.
 * - No CPU fallback: without a CUDA device fftmech_create fails.
 * - Batches: a context made by fftmech_create_batched holds B problems of
 *   the same grid (independent RVEs, e.g. one per macroscale point, Sec. 3.2).
 *   Every field argument then holds the B problems back to back (problem b's
 *   scalar fields at offset b N, its d-component fields at b d N, with N the
 *   voxels of one problem), every `info` argument is an array of B records
 *   (3 B for the staggered step, problem-major), and each problem converges
 *   on its own: its iterations stop when it has, while the others continue.
 */
#ifndef FFTMECH_H
#define FFTMECH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFTMECH_OK = 0,
  FFTMECH_ERR_INVALID_ARG = 1,
  FFTMECH_ERR_UNSUPPORTED_SIZE = 2, /* grid size not 2^a 3^b in [2, 4096], or dim unsupported */
  FFTMECH_ERR_NOT_CONVERGED = 3,    /* PCG hit max_iter before tol */
  FFTMECH_ERR_NONFINITE = 4,        /* NaN/Inf residual or breakdown */
  FFTMECH_ERR_TIMEOUT = 5,          /* reserved: the library has no device-side waits (its loops
                                       are conditional graph nodes bounded by max_iter), so no
                                       call returns it */
  FFTMECH_ERR_CUDA = 6,
  FFTMECH_ERR_OOM = 7
} fftmech_status;

typedef enum {
  FFTMECH_FP64 = 0,  /* every field, FFT and stencil in double */
  FFTMECH_MIXED = 1  /* float fields, FFTs and stencils; double iterates, dot products,
                        averages and periodic true-residual replacement */
} fftmech_precision;

/* Grid. dim = 2 or 3; n[0] = nx, n[1] = ny, n[2] = nz (n[2] = 1 in 2D).
 * h: voxel size for mechanics and the phase field; h_diff: voxel size for
 * diffusion (the paper's diffusion runs in its own units). */
typedef struct {
  int dim;
  int n[3];
  double h;
  double h_diff;
} fftmech_grid;

/* Phase properties (Sec. 3) and model constants.
 * E, nu: Young's modulus and Poisson ratio of each phase (plane strain in 2D).
 * D_solid, D_pore: diffusivities (Sec. 2.1). Gc, l0: fracture energy and
 * regularisation length (Eq. crack). kappa: residual stiffness in
 * g(d) = (1 - d)^2 + kappa (Sec. 2.4). S_sol, M_ppt: solubility limit and
 * molar volume of the precipitate (Sec. 2.2, Eq. eigen-simplify). */
typedef struct {
  double E_solid, nu_solid, E_pore, nu_pore;
  double D_solid, D_pore;
  double Gc, l0, kappa;
  double S_sol, M_ppt;
} fftmech_materials;

/* PCG controls. Stop when the gradient-space residual norm (the paper's CG
 * residual, equal to sqrt(r.M^-1 r) of the potential PCG) has dropped by
 * `tol` relative to that of the right-hand side, or after max_iter
 * iterations (status NOT_CONVERGED).
 * replace_residual (MIXED only, 0/1): reliable updates; after every 16th
 * iteration the device checks whether r.M^-1 r has fallen 100-fold since
 * the last replacement and, if so, replaces the float recursive residual by
 * the true residual b - K u in the next iteration (search direction kept;
 * the problems of a batch due at that point are replaced together). The
 * true residual is evaluated in double-float arithmetic (about 2^-48
 * relative per operation) from the double-float iterate. After
 * convergence of the float recursion the true residual is
 * checked; a problem whose true residual misses tol continues from it (at
 * most three times).
 * Every decision of the loop is taken on the device. execution:
 * FFTMECH_EXEC_GRAPH (0, default) runs each call as one CUDA graph whose
 * loops are conditional nodes (no host synchronisation inside a solve or a
 * staggered step; the graph is captured on the first call and re-captured
 * when the arguments change); FFTMECH_EXEC_HOST runs the same kernels with
 * the host driving the loops, reading the device's decisions after every
 * iteration (slower; used with per-launch profiling). Both give
 * bit-identical results. check_every is not used (kept for the layout).
 * launch_mode: bit 0 clear (default) launches the kernels of a PCG
 * iteration as programmatic dependent launches (each kernel starts
 * launching while the previous one finishes and waits on the device for
 * its results), set uses plain stream order (bit-identical results). Bit 1
 * set runs, on 2D grids of up to 2^21 voxels per launch, the direction and
 * the next iteration's stencil as one kernel (the same iterates up to the
 * summation order of <p, K p>); clear (default) keeps them apart.
 * fftmech_autotune times both and its choice then replaces bit 1.
 * precond: preconditioner of the equilibrium PCG. FFTMECH_PRECOND_LAPLACE
 * (0, default): F^-1 (1 / |D|^2) F per component, the projection of App. A
 * (Eq. g-42). FFTMECH_PRECOND_REFERENCE (1): the inverse of the Galerkin
 * operator of a homogeneous isotropic reference medium, per mode the d x d
 * Hermitian matrix |D|^2 I + rho conj(D) D^T + D conj(D)^T inverted (2D in
 * the column pass, 3D in the z pass), with rho = lambda / mu of the solid
 * (the Moulinec-Suquet reference medium the paper names as the classical
 * scheme's preconditioner, Sec. 1; exact for a homogeneous medium of that
 * Poisson ratio). Same solution, fewer iterations; diffusion and
 * phase-field solves keep the Laplace one. */
enum { FFTMECH_EXEC_GRAPH = 0, FFTMECH_EXEC_HOST = 1 };
enum { FFTMECH_PRECOND_LAPLACE = 0, FFTMECH_PRECOND_REFERENCE = 1 };
typedef struct {
  double tol;
  int max_iter;
  int replace_residual;
  int check_every;
  int launch_mode;
  int execution;
  int precond;
} fftmech_solver_opts;

/* Per-solve report (host struct). All averages in FP64 over every voxel. */
typedef struct {
  int status;               /* fftmech_status of the solve */
  int iters;                /* PCG iterations (operator applications) */
  double rel_res;           /* final recursive relative residual */
  double true_rel_res;      /* FP64 true relative residual of the returned iterate */
  double mean_stress[6];    /* <sigma>, Voigt */
  double mean_strain[6];    /* <eps>, Voigt (equals eps_mac up to rounding) */
  double mean_flux[3];      /* <j> of the diffusion step (HOMOGENISE) */
  double mean_c;            /* <c> after the diffusion step */
  double porosity;          /* eta = |Omega_p| / |Omega| */
  double elastic_energy;    /* sum 1/2 (eps - e I) : sigma h^dim */
  double total_damage;      /* sum of d over the voxels */
  double frac_damaged;      /* fraction of solid voxels with d > 0.9 */
  double device_ms;         /* device time of the solve (CUDA events on the context stream) */
} fftmech_solve_info;

typedef struct fftmech_ctx fftmech_ctx;

/* Create a context for one grid. `stream` is a cudaStream_t (NULL = a new
 * stream owned by the context). Allocates the workspace (about 60 bytes per
 * voxel for MIXED 2D, about 100 for MIXED 3D) on the current CUDA device.
 * Returns INVALID_ARG for bad pointers or materials, UNSUPPORTED_SIZE for a
 * grid dimension that is not 2^a 3^b (at most 2187 for powers of three,
 * 2048 for powers of two and mixed sizes within the same per-line limits;
 * in 3D every n >= 2 and x lines short enough for the brick kernels' shared
 * memory) or dim not in {2, 3}, OOM if the workspace does not fit, CUDA if
 * no device is usable. */
fftmech_status fftmech_create(fftmech_ctx** ctx, const fftmech_grid* grid,
                              const fftmech_materials* mat, fftmech_precision precision,
                              const fftmech_solver_opts* opts, void* stream);

/* A context for `batch` >= 1 independent problems of the same grid, solved
 * together (every kernel launch covers all of them; grid.y = problem).
 * The workspace grows linearly with batch. fftmech_create(...) equals
 * fftmech_create_batched(..., 1, ...). */
fftmech_status fftmech_create_batched(fftmech_ctx** ctx, const fftmech_grid* grid, int batch,
                                      const fftmech_materials* mat, fftmech_precision precision,
                                      const fftmech_solver_opts* opts, void* stream);

/* Number of problems of a context (0 for NULL). */
int fftmech_batch_size(const fftmech_ctx* ctx);

/* Free the workspace (and the stream, if the context created it). */
fftmech_status fftmech_destroy(fftmech_ctx* ctx);

/* Replace the solver options of an existing context. */
fftmech_status fftmech_set_solver_opts(fftmech_ctx* ctx, const fftmech_solver_opts* opts);

/* Human-readable name of a status code, and the last error message of a
 * context (empty string if none). Both strings are owned by the library. */
const char* fftmech_status_string(int status);
const char* fftmech_last_error(const fftmech_ctx* ctx);

enum { FFTMECH_DIFF_NONE = 0, FFTMECH_DIFF_HOMOGENISE = 1, FFTMECH_DIFF_TRANSIENT = 2 };
enum { FFTMECH_EIG_FROM_PRECIPITATE = 0, FFTMECH_EIG_PRESCRIBED = 1 };

/* Diffusion step (Sec. 2.1; Algorithm 1, "Diffusion of chemical species").
 * mode FFTMECH_DIFF_HOMOGENISE (the paper): solves div j = 0,
 *   j = -D(x) grad c, <grad c> = grad_c_mac (Eqs. diffusion, diffusion-final)
 *   for the fluctuation phi (Eq. micro-gradient), then writes
 *   c = grad_c_mac . x + phi + beta with beta_pore / beta_solid of
 *   Eq. (psi-two-values), so <c>_pore = c_macro / eta and <c>_solid = 0
 *   (Eq. concentration-correct). x is the voxel position k * h_diff.
 *   dt, dirichlet_mask, dirichlet_value are ignored; c is output only.
 *   info->mean_flux = <j>.
 * mode FFTMECH_DIFF_TRANSIENT (an extension, not in the paper, whose RVE
 *   diffusion is steady): one backward-Euler step of
 *   dc/dt = div(D(x) grad c) with the same forward-difference Galerkin
 *   operator; voxels with dirichlet_mask != 0 are held at dirichlet_value.
 *   c is the concentration at the old time on input, the new one on output.
 * phase: uint8 [N]; c: double [N]; dirichlet_mask: uint8 [N] or NULL. */
fftmech_status fftmech_diffusion_step(fftmech_ctx* ctx, const uint8_t* phase, int mode,
                                      const double grad_c_mac[3], double c_macro, double dt,
                                      const uint8_t* dirichlet_mask, double dirichlet_value,
                                      double* c, fftmech_solve_info* info);

/* Mechanical equilibrium with eigenstrain (Sec. 2.3; Algorithm 1,
 * "Development of stresses"): div[g(d) C(x) : (eps - e I)] = 0 with
 * <eps> = eps_mac (Eqs. solid, solid-final), C(x) = omega C_solid +
 * (1 - omega) C_pore isotropic, g(d) = (1 - d)^2 + kappa (Sec. 2.4),
 * isotropic eigenstrain e(x) I (Eq. eigen-simplify; in-plane identity in 2D
 * plane strain).
 * phase: uint8 [N]; eig: field [N] (NULL = 0); damage: double [N] (NULL = 0);
 * eps_mac: Voigt (3 used in 2D, 6 in 3D); u: double [dim * N], the
 * displacement fluctuation: warm start on input (zero-mean), solution on
 * output; strain, stress: field [nv * N] outputs (NULL = not written),
 * strain = eps_mac + sym grad+ u, stress = g C : (strain - e I).
 * info: iterations, residuals, <sigma>, <eps>, elastic energy. */
fftmech_status fftmech_equilibrium_solve(fftmech_ctx* ctx, const uint8_t* phase, const void* eig,
                                         const double* damage, const double eps_mac[6], double* u,
                                         void* strain, void* stress, fftmech_solve_info* info);

/* History update and phase-field solve (Sec. 2.4; Algorithm 1, "Crack
 * initiation and propagation"). First H = max(H, psi+(strain - e I))
 * with psi+ of Eq. (energy) (undegraded phase Lame constants; in 3D the bulk
 * factor lambda + 2 mu / 3 and the 3D deviator), then solves
 * (Gc / (2 l0) + H) d - (Gc l0 / 2) div grad d = H (Eqs. crack, crack-fft) with
 * the Laplacian's symbol read as -|D|^2 (symmetric positive definite).
 * strain: field [nv * N]; eig: field [N] (NULL = 0); phase: uint8 [N];
 * H: field [N] in/out; damage: double [N], warm start in, solution out.
 * info: iterations, residuals, total damage, fraction of damaged solid. */
fftmech_status fftmech_phasefield_solve(fftmech_ctx* ctx, const void* strain, const void* eig,
                                        const uint8_t* phase, void* H, double* damage,
                                        fftmech_solve_info* info);

/* State carried across staggered steps (all caller-owned, N voxels). */
typedef struct {
  const uint8_t* phase; /* uint8 [N] */
  double* c;            /* concentration, double [N] */
  void* c_ppt;          /* precipitate concentration, field [N] (NULL = not kept) */
  void* eig;            /* eigenstrain e(x), field [N] */
  double* u;            /* displacement fluctuation, double [dim * N] */
  void* strain;         /* field [nv * N] */
  void* stress;         /* field [nv * N] */
  void* H;              /* history field, field [N] */
  double* damage;       /* phase field d, double [N] */
} fftmech_state;

/* Loads of one staggered step.
 * diffusion_mode: FFTMECH_DIFF_*; the HOMOGENISE / TRANSIENT inputs as in
 * fftmech_diffusion_step. eig_mode FFTMECH_EIG_FROM_PRECIPITATE:
 * c_ppt = (c - S_sol)_+ and e = (c_ppt M_ppt - 1)_+ in the pores, 0 in the
 * solid (Sec. 2.2); FFTMECH_EIG_PRESCRIBED: e = eig_scale * eig_field
 * (eig_field: field [N]). eps_mac: macro strain (Voigt).
 * c_macro_each / grad_c_mac_each (HOMOGENISE, optional; device memory, read
 * when the step runs): per-problem macro concentration [B] and gradient
 * [3 * B] of a batch, replacing c_macro and grad_c_mac (a macroscale
 * driver gives each RVE its material point's c(X) and grad c(X), Sec. 3.2;
 * new values need no re-capture of the step's graph). NULL: the scalars for
 * every problem. info.mean_c reports each problem's c_macro. */
typedef struct {
  int diffusion_mode;
  double grad_c_mac[3];
  double c_macro;
  double dt;
  const uint8_t* dirichlet_mask;
  double dirichlet_value;
  int eig_mode;
  const void* eig_field;
  double eig_scale;
  double eps_mac[6];
  const double* c_macro_each;
  const double* grad_c_mac_each;
} fftmech_step_params;

/* One staggered load step in Algorithm 1's order (Sec. 2.5): diffusion ->
 * precipitation -> eigenstrain -> equilibrium (stiffness degraded by the
 * damage of the previous step) -> history -> phase field. The degradation
 * by the new damage (Algorithm 1, last line) takes effect in the next call.
 * info[3 b + 0] = diffusion, info[3 b + 1] = equilibrium, info[3 b + 2] =
 * phase field of problem b (3 records per problem of the batch). The step
 * parameters are shared by the problems of a batch. */
fftmech_status fftmech_staggered_step(fftmech_ctx* ctx, fftmech_state* state,
                                      const fftmech_step_params* params,
                                      fftmech_solve_info* info);

/* Asynchronous staggered step: enqueues the same work as
 * fftmech_staggered_step on the context's stream and returns without
 * waiting. Every pointer of `state` and `params` must be device memory
 * (INVALID_ARG otherwise); nothing is allocated, staged or copied, and the
 * host does not synchronise. If the stream is being captured (stream
 * capture into the caller's own CUDA graph), the step is emitted into that
 * graph, conditional nodes included, and runs whenever the caller launches
 * it. The reports of the step are written on the device and copied to
 * library-owned pinned memory at its end; read them with fftmech_step_info.
 * No counterpart in the paper. */
fftmech_status fftmech_staggered_step_async(fftmech_ctx* ctx, const fftmech_state* state,
                                            const fftmech_step_params* params);

/* Reports of the last staggered step enqueued on the context (by
 * fftmech_staggered_step, fftmech_staggered_step_async, or a replay of a
 * graph that captured it): synchronises the context's stream, then fills
 * info[3 B] as fftmech_staggered_step does and returns the first solver
 * status that is not OK. INVALID_ARG if no step was enqueued. */
fftmech_status fftmech_step_info(fftmech_ctx* ctx, fftmech_solve_info* info);

/* Gradient of an objective of the staggered solve with respect to the
 * per-voxel eigenstrain field (an extension: the paper solves forward
 * only). Forward model: `steps` staggered steps (Algorithm 1, Sec. 2.5)
 * without diffusion, the eigenstrain prescribed as e_s(x) = ramp[s] e(x)
 * (Eq. eigen-simplify's isotropic eigenstrain), the fixed macro strain
 * eps_mac (Voigt, NULL = 0), H and d starting at 0. Objective at the last
 * step: FFTMECH_OBJ_ENERGY, the total elastic energy
 * sum 1/2 (eps - e I) : sigma h^dim; FFTMECH_OBJ_DAMAGE, the summed damage
 * sum d. J receives its value and grad[N] (double, device) dJ/de(x), by the
 * discrete adjoint: per step backwards, a phase-field adjoint solve
 * (Eq. crack-fft's operator), the derivative through the history max
 * (where psi+ >= H_prev, ties to psi+) and psi+ of Eq. (energy) (the
 * derivative of [x]_+ is 1 for x > 0, else 0), an equilibrium adjoint solve
 * (a PCG on the same operator K = grad+^T g C grad+ with the right-hand side
 * grad+^T tau), and the explicit dependences on e and on the previous
 * damage through g(d). Checkpoints of (H, d, u) every `checkpoint_every`
 * steps; each segment is recomputed forward before its reverse steps.
 * phase: uint8 [N], e_field: field [N], grad: double [N], all device
 * memory; ramp[steps] on the host. One problem per context (batch 1).
 * Allocates its checkpoint and work buffers for the call (about
 * (20 + 28 n_ckpt + 24 checkpoint_every) bytes per voxel in MIXED 2D).
 * info_last (3 records, NULL = none): the forward's last step. Returns the
 * first solver status that is not OK, else OK. */
enum { FFTMECH_OBJ_ENERGY = 0, FFTMECH_OBJ_DAMAGE = 1 };
fftmech_status fftmech_adjoint_eigenstrain(fftmech_ctx* ctx, const uint8_t* phase, const void* e_field, int steps,
                                           const double* ramp, const double eps_mac[6], int objective,
                                           int checkpoint_every, double* grad, double* J,
                                           fftmech_solve_info* info_last);

/* Launch-shape autotuner (no counterpart in the paper). Times `iterations`
 * equilibrium PCG iterations on a synthetic two-phase field of the
 * context's grid and batch (graph execution, best of two runs per
 * candidate) for candidate launch shapes: column strip width and stencil
 * strip rows (2D), stencil brick depth (3D), stencil blocks per problem,
 * lines per block of the x-line kernels and, on 2D grids of up to 2^21
 * voxels per launch, split or fused direction and stencil kernels (with
 * the fused kernel's rows per block), one parameter at a time from the
 * best so far. Applies the fastest and keeps it for the process: a later
 * call on another context of the same device, grid, batch and precision
 * applies it without timing (the description then ends in "(cached)"; the
 * times are those of the original tuning). New contexts always start from
 * the rule-based shapes. Reports the time per iteration before and after
 * (microseconds) and a description of the shapes (owned by the context).
 * Allocates temporary device buffers; results of later solves change only
 * within rounding (the reductions' block partitions change).
 * iterations = 0 only reports the shapes in use. */
fftmech_status fftmech_autotune(fftmech_ctx* ctx, int iterations, double* before_us, double* after_us,
                                const char** choice);

/* Applies launch shapes given as the description fftmech_autotune returns
 * ("L_dir=2 L_upd=1 ty=8 zc=1 grid=1216 cols=4 L_ds=0": any subset of these
 * keys, separated by spaces; a trailing "(cached)" is ignored), so that a
 * tuning can be kept across processes. Keys left out keep their values.
 * L_ds = 0 selects the split direction and stencil kernels, L_ds > 0 the
 * fused kernel with that many rows per block. Returns INVALID_ARG (and
 * changes nothing) for an unknown key or a shape the grid cannot take. */
fftmech_status fftmech_set_launch_shapes(fftmech_ctx* ctx, const char* shapes);

/* Homogenised RVE diffusion (Sec. 2.1: Eqs. diffusion, diffusion-final,
 * phi-fft) with a choice of gradient operator (Sec. 2.6, the comparison of
 * Fig. 2): FFTMECH_GRAD_FORWARD (e^{i theta} - 1) / h, the operator of every
 * other call; FFTMECH_GRAD_CENTRAL i sin(theta) / h (the garbled printed
 * formula read as the central difference); FFTMECH_GRAD_CENTRAL8 the
 * 8th-order central difference (coefficients from the moment conditions:
 * 4/5, -1/5, 4/105, -1/280); FFTMECH_GRAD_FOURIER i xi (odd grid sizes only:
 * UNSUPPORTED_SIZE otherwise). The Galerkin system D^H kappa(x) D phi =
 * -D^H kappa(x) G is solved by PCG on the spectrum of phi with the
 * preconditioner 1 / |D|^2 (0 where D vanishes), the operator applied by one
 * inverse and one forward transform of the gradient per iteration. FP64
 * whatever the context's precision; host-driven; one problem per context;
 * allocates temporary device buffers. Uses the context's grid, h_diff,
 * D_pore, D_solid, tol and max_iter. phase: uint8 [N]; grad_c_mac: the macro
 * gradient; phi: double [N] (zero mean) or NULL; grad_c = G + D phi:
 * double [dim N] or NULL (device pointers). info: iterations, residual,
 * mean flux <j> = -<kappa grad c>. */
enum { FFTMECH_GRAD_FORWARD = 0, FFTMECH_GRAD_CENTRAL = 1, FFTMECH_GRAD_CENTRAL8 = 2, FFTMECH_GRAD_FOURIER = 3 };
/* OR'ed into the gradient of fftmech_phasefield_operator: the printed
 * phase-field Laplacian read literally (see there). */
enum { FFTMECH_PF_LITERAL = 256 };
fftmech_status fftmech_homogenise_operator(fftmech_ctx* ctx, const uint8_t* phase, int gradient,
                                          const double grad_c_mac[3], double* phi, double* grad_c,
                                          fftmech_solve_info* info);

/* Mechanical equilibrium with a choice of gradient operator (Sec. 2.6
 * applied to Eqs. solid and solid-final; the stress panels of Fig. 2):
 * D^H F[g C : F^-1(sym D u)] = -D^H F[g C : (E - e I)] solved by PCG on the
 * displacement spectra with the preconditioner 1 / |D|^2 per component,
 * gradient one of FFTMECH_GRAD_* (FOURIER: odd grid sizes only). FP64
 * whatever the context's precision; host-driven; one problem per context;
 * allocates temporary device buffers. Uses the context's grid, h, the
 * elastic constants, kappa, tol and max_iter. phase: uint8 [N]; eig:
 * double [N] or NULL (0); damage: double [N] or NULL (g = 1), g = (1 -
 * d)^2 + kappa; eps_mac: Voigt (tensor shears); strain = E + sym D u and
 * stress = g C : (strain - e I): double [nv N] or NULL (device pointers).
 * info: iterations, residual, <sigma>, <eps>. */
fftmech_status fftmech_equilibrium_operator(fftmech_ctx* ctx, const uint8_t* phase, const double* eig,
                                            const double* damage, const double eps_mac[6], int gradient,
                                            double* strain, double* stress, fftmech_solve_info* info);

/* History update and AT2 phase field with a choice of gradient operator
 * (Eqs. energy, crack and crack-fft with the symbol of Sec. 2.6; the damage
 * panels of Fig. 2): H = max(H, psi+(strain - e I)), then
 * (a + H) d + b F^-1(|D|^2 F d) = H, a = Gc / (2 l0), b = Gc l0 / 2, by
 * PCG on the spectrum of d with the preconditioner 1 / (a + <H> + b |D|^2),
 * gradient one of FFTMECH_GRAD_* (FOURIER: odd grid sizes only). FP64;
 * host-driven; one problem per context; allocates temporary device
 * buffers. phase: uint8 [N]; strain: double [nv N] (Voigt, tensor shears);
 * eig: double [N] or NULL; H: double [N], updated in place; d: double [N]
 * output (device pointers). info: iterations, residual, total_damage (the
 * sum of d over the voxels). gradient | FFTMECH_PF_LITERAL reads the
 * printed Laplacian "i xi . i xi" literally as sum_a D_a^2 (for the forward
 * difference a non-symmetric one-sided second difference):
 * (a + H) d - b F^-1(sum_a D_a^2 F d) = H, solved by restarted GMRES(40)
 * (as the paper solves it) with the preconditioner above on the right;
 * iterations then counts GMRES steps. */
fftmech_status fftmech_phasefield_operator(fftmech_ctx* ctx, const uint8_t* phase, const double* strain,
                                           const double* eig, int gradient, double* H, double* d,
                                           fftmech_solve_info* info);

/* Element offset of problem `problem`'s segment in a field with
 * `components` components per voxel (1 for scalar fields, dim for u, 3 or
 * 6 for strain and stress) of a batched context: problem * components * N. */
fftmech_status fftmech_problem_offset(const fftmech_ctx* ctx, int problem, int components, long long* offset);

/* Graph execution counters of a context: graphs captured (or re-captured
 * after an argument change), graph launches, and the kernels those
 * launches ran (counted when a call's reports are read: each conditional
 * body's launches times its executions, from the solves' iteration,
 * replacement and restart counts; for a batch the largest count of its
 * problems). disabled = 1 when a graph failed to build or launch and the
 * context fell back to host-driven execution, with the reason in *reason
 * (owned by the library). Any pointer may be NULL. */
fftmech_status fftmech_graph_stats(const fftmech_ctx* ctx, long long* builds, long long* launches,
                                   long long* kernels, int* disabled, const char** reason);

/* A group of contexts stepped together: a batch of uneven grids is one
 * uniform-batch context per grid size (Sec. 3.2 treats every RVE as an
 * independent problem), and the group runs the staggered steps of all of
 * them as ONE CUDA graph, one parallel branch per context, each branch with
 * its own device-driven loops; one graph launch per step, no host thread
 * per context and no host synchronisation inside the step. The graph is
 * captured on the first fftmech_group_step and again when the arguments
 * change. Contexts must be distinct, on one device, with distinct streams
 * (used only while capturing); `stream` (NULL = a new stream owned by the
 * group) is where the graph runs. No counterpart in the paper. */
typedef struct fftmech_group fftmech_group;
fftmech_status fftmech_group_create(fftmech_group** group, fftmech_ctx* const* ctxs, int n, void* stream);
fftmech_status fftmech_group_destroy(fftmech_group* group);
/* One staggered step of every context of the group. states[i], params[i]
 * and infos[i] (3 * fftmech_batch_size(ctxs[i]) records) belong to
 * context i; every pointer must be device memory (INVALID_ARG otherwise).
 * Returns after the step has completed: INVALID_ARG or CUDA on failure
 * (fftmech_group_last_error gives the message), else the first solver
 * status that is not OK. */
fftmech_status fftmech_group_step(fftmech_group* group, const fftmech_state* const* states,
                                  const fftmech_step_params* const* params, fftmech_solve_info* const* infos);
/* Graphs captured, graph launches and the kernels they ran. */
fftmech_status fftmech_group_stats(const fftmech_group* group, long long* builds, long long* launches,
                                   long long* kernels);
const char* fftmech_group_last_error(const fftmech_group* group);

/* Staggered steps of several contexts at once: a group made for this call
 * (the graph is captured every time; keep a group to reuse it). Same
 * arguments and results as fftmech_group_step. No counterpart in the paper. */
fftmech_status fftmech_staggered_step_many(fftmech_ctx* const* ctxs, int n, fftmech_state* const* states,
                                           const fftmech_step_params* const* params,
                                           fftmech_solve_info* const* infos);

/* Macroscale bar of the multiscale diffusion (Sec. 3.2): a bar along X whose
 * face X = 0 (the steel-concrete interface) takes a constant influx
 * `flux_in` and whose far end is closed, coupled to the M RVEs of a batched
 * context (M = fftmech_batch_size(ctx)). The paper does not give its
 * finite-difference scheme; this one: nodes X_m = m dX (m = 0 .. M,
 * dX = length / M) hold the macro concentration c_m in device memory;
 * element e (nodes e, e + 1) carries RVE e at its midpoint, which receives
 * grad c_mac = ((c_{e+1} - c_e) / dX, 0, 0) along its x axis and
 * c_macro = (c_e + c_{e+1}) / 2; lumped masses w = dX inside and dX / 2 at
 * the ends, forward Euler
 *   c_m += dt / w_m (J_{m-1/2} - J_{m+1/2}),  J_{e+1/2} = <j_x> of RVE e,
 *   J_{-1/2} = flux_in, J_{M+1/2} = 0.
 * length is in the RVE's length unit (h_diff per voxel); dt must satisfy
 * dt <= dX^2 / (2 max(D_pore, D_solid)) (INVALID_ARG otherwise).
 * c0: M + 1 host values (NULL = 0). The bar owns M + 1 + 4 M doubles of
 * device memory. */
typedef struct fftmech_bar fftmech_bar;
fftmech_status fftmech_bar_create(fftmech_bar** bar, fftmech_ctx* ctx, double length, double dt, double flux_in,
                                  const double* c0);
fftmech_status fftmech_bar_destroy(fftmech_bar* bar);
/* One macro time step: the element inputs from c^n, one staggered step of
 * all RVEs (Algorithm 1 with diffusion_mode HOMOGENISE and the per-element
 * c_macro / grad c_mac; the other fields of `params` as in
 * fftmech_staggered_step: eigenstrain mode, eps_mac, ...), then c^{n+1}
 * from the RVEs' mean fluxes, all enqueued on the context's stream as one
 * CUDA graph (captured on the first call). state: device pointers of the
 * batch. info: 3 M records as fftmech_staggered_step fills them (mean_flux
 * and mean_c of each RVE in its diffusion record). */
fftmech_status fftmech_bar_step(fftmech_bar* bar, const fftmech_state* state, const fftmech_step_params* params,
                                fftmech_solve_info* info);
/* Nodal concentrations c_0 .. c_M to / from host memory. */
fftmech_status fftmech_bar_read(const fftmech_bar* bar, double* c_host);
fftmech_status fftmech_bar_write(fftmech_bar* bar, const double* c_host);

/* Instrumentation (no counterpart in the paper): kernel classes of the PCG
 * loop. When profiling is enabled, every launch of a class is bracketed by
 * CUDA events on the context's stream and its duration accumulated; launch
 * counts are kept whether or not profiling is on. */
enum {
  FFTMECH_K_DIRECTION = 0, /* x-line IFFT + new search direction (2D fused: + q = K p) */
  FFTMECH_K_UPDATE = 1,    /* iterate / residual update + x-line FFT */
  FFTMECH_K_COLUMN = 2,    /* y (and z) line FFTs, Fourier multiplier, <r, M^-1 r>, inverse */
  FFTMECH_K_RESIDUAL = 3,  /* true residual + x-line FFT */
  FFTMECH_K_OTHER = 4,     /* pointwise and post-processing kernels */
  FFTMECH_K_STENCIL = 5,   /* q = K p and <p, K p> (stencil tiles) */
  FFTMECH_K_COUNT = 6
};

/* Enable (1) or disable (0) per-launch event timing; resets the counters. */
fftmech_status fftmech_profile_enable(fftmech_ctx* ctx, int enable);

/* Launches and summed device time (ms) of one kernel class since the last
 * fftmech_profile_enable; kclass = FFTMECH_K_COUNT gives the totals over
 * all classes. total_ms is 0 while profiling is disabled. */
fftmech_status fftmech_profile_read(fftmech_ctx* ctx, int kclass, long long* launches,
                                    double* total_ms);

/* Stand-alone complex-to-complex FFT with the library's Stockham kernels
 * (the transform every solve uses; exposed for testing and comparison).
 * data: interleaved complex, device memory, C order with n[0] points per
 * line: one line (ndim = 1), n[1] rows (ndim = 2) or n[2] planes of n[1]
 * rows (ndim = 3), transformed in place along every axis. The twiddle
 * tables of a length are made on its first use on a device and kept until
 * the process exits.
 * precision: FFTMECH_FP64 (complex double) or FFTMECH_MIXED (complex
 * float). inverse = 0: X[k] = sum_j x[j] exp(-2 pi i jk/n); inverse = 1: the
 * same with +i and no 1/n factor. stream: cudaStream_t (NULL = default).
 * Synchronises the stream before returning. */
fftmech_status fftmech_fft(int ndim, const int n[3], int precision, int inverse, void* data,
                           void* stream);

/* Allocation-free variant of fftmech_fft. The paper has no counterpart: it
 * exists for callers that must not allocate device memory themselves or
 * through this library, e.g. code that runs while other streams must keep
 * running (cudaMalloc and cudaFree can synchronise the whole device), code
 * whose device memory belongs to another allocator or to a fixed budget (a
 * framework's memory pool, where a raw cudaMalloc can fail or fragment the
 * pool), or code that must not meet an out-of-memory error in mid-run.
 * fftmech_fft allocates the twiddle tables of every new length it meets;
 * this entry point keeps them in one fixed device array inside the library
 * instead (about
 * 103 KiB, held on every GPU that loads the library until the process exits)
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 * Same arguments, layout and results as fftmech_fft, with each n[i] at most
 * FFTMECH_FFT_NOALLOC_MAX_N; larger sizes return
 * FFTMECH_ERR_UNSUPPORTED_SIZE before any work.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current). No call may be made while `stream` is
 * being captured into a CUDA graph (or, in global capture mode, while any
 * stream is): every call copies from a host buffer and synchronises
 * `stream`, which a capture does not allow (the capture would be
 * invalidated). All calls share the array and it keeps the last call's
 * twiddles: two calls whose transforms overlapped on the GPU would race, so
 * calls are serialised by a process-wide lock and each returns only after
 * its copies and transform have completed on `stream` (also when it returns
 * an error). */
#define FFTMECH_FFT_NOALLOC_MAX_N 2187
fftmech_status fftmech_fft_noalloc(int ndim, const int n[3], int precision, int inverse,
                                   void* data, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFTMECH_H */
