"""ctypes binding of libfftmech (include/fftmech.h): the same entry points,
structs and constants, argument marshalling only. Every computation runs in
the CUDA library; there is no Python or CPU fallback, and loading fails
loudly when the library has not been built.

Buffers may be torch CUDA tensors (passed by data_ptr()), numpy arrays or
host torch tensors (passed as host pointers; the library stages them through
device memory), or raw integer addresses.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfftmech.so")

# status codes
FFTMECH_OK = 0
FFTMECH_ERR_INVALID_ARG = 1
FFTMECH_ERR_UNSUPPORTED_SIZE = 2
FFTMECH_ERR_NOT_CONVERGED = 3
FFTMECH_ERR_NONFINITE = 4
FFTMECH_ERR_TIMEOUT = 5
FFTMECH_ERR_CUDA = 6
FFTMECH_ERR_OOM = 7
# precisions
FFTMECH_FP64 = 0
FFTMECH_MIXED = 1
# diffusion / eigenstrain modes
FFTMECH_DIFF_NONE = 0
FFTMECH_DIFF_HOMOGENISE = 1
FFTMECH_DIFF_TRANSIENT = 2
FFTMECH_EIG_FROM_PRECIPITATE = 0
FFTMECH_EIG_PRESCRIBED = 1
# execution of a solve or a staggered step
FFTMECH_EXEC_GRAPH = 0
FFTMECH_EXEC_HOST = 1
# gradient operators (fftmech_*_operator)
FFTMECH_GRAD_FORWARD = 0
FFTMECH_GRAD_CENTRAL = 1
FFTMECH_GRAD_CENTRAL8 = 2
FFTMECH_GRAD_FOURIER = 3
FFTMECH_PF_LITERAL = 256  # phase field: the printed Laplacian read literally (GMRES)
# preconditioner of the equilibrium PCG
FFTMECH_PRECOND_LAPLACE = 0
FFTMECH_PRECOND_REFERENCE = 1
# objectives of the eigenstrain adjoint
FFTMECH_OBJ_ENERGY = 0
FFTMECH_OBJ_DAMAGE = 1
# kernel classes (instrumentation)
FFTMECH_K_DIRECTION = 0
FFTMECH_K_UPDATE = 1
FFTMECH_K_COLUMN = 2
FFTMECH_K_RESIDUAL = 3
FFTMECH_K_OTHER = 4
FFTMECH_K_STENCIL = 5
FFTMECH_K_COUNT = 6
KERNEL_CLASS_NAMES = ["direction", "update", "column", "residual", "other", "stencil"]

c_double3 = ctypes.c_double * 3
c_double6 = ctypes.c_double * 6
c_int3 = ctypes.c_int * 3


class fftmech_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", c_int3), ("h", ctypes.c_double),
                ("h_diff", ctypes.c_double)]


class fftmech_materials(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("E_solid", "nu_solid", "E_pore", "nu_pore", "D_solid", "D_pore",
                 "Gc", "l0", "kappa", "S_sol", "M_ppt")]


class fftmech_solver_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("replace_residual", ctypes.c_int), ("check_every", ctypes.c_int),
                ("launch_mode", ctypes.c_int), ("execution", ctypes.c_int), ("precond", ctypes.c_int)]


class fftmech_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("mean_stress", c_double6), ("mean_strain", c_double6),
                ("mean_flux", c_double3), ("mean_c", ctypes.c_double),
                ("porosity", ctypes.c_double), ("elastic_energy", ctypes.c_double),
                ("total_damage", ctypes.c_double), ("frac_damaged", ctypes.c_double),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class fftmech_state(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_void_p), ("c", ctypes.c_void_p), ("c_ppt", ctypes.c_void_p),
                ("eig", ctypes.c_void_p), ("u", ctypes.c_void_p), ("strain", ctypes.c_void_p),
                ("stress", ctypes.c_void_p), ("H", ctypes.c_void_p), ("damage", ctypes.c_void_p)]


class fftmech_step_params(ctypes.Structure):
    _fields_ = [("diffusion_mode", ctypes.c_int), ("grad_c_mac", c_double3),
                ("c_macro", ctypes.c_double), ("dt", ctypes.c_double),
                ("dirichlet_mask", ctypes.c_void_p), ("dirichlet_value", ctypes.c_double),
                ("eig_mode", ctypes.c_int), ("eig_field", ctypes.c_void_p),
                ("eig_scale", ctypes.c_double), ("eps_mac", c_double6),
                ("c_macro_each", ctypes.c_void_p), ("grad_c_mac_each", ctypes.c_void_p)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libfftmech.so (built by paper_2305_13081_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libfftmech.so not found at {path}: build it with "
            "`python -m paper_2305_13081_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    i = ctypes.c_int
    d = ctypes.c_double
    sigs = {
        "fftmech_create": (i, [P(vp), P(fftmech_grid), P(fftmech_materials), i,
                               P(fftmech_solver_opts), vp]),
        "fftmech_create_batched": (i, [P(vp), P(fftmech_grid), i, P(fftmech_materials), i,
                                       P(fftmech_solver_opts), vp]),
        "fftmech_batch_size": (i, [vp]),
        "fftmech_destroy": (i, [vp]),
        "fftmech_set_solver_opts": (i, [vp, P(fftmech_solver_opts)]),
        "fftmech_status_string": (ctypes.c_char_p, [i]),
        "fftmech_last_error": (ctypes.c_char_p, [vp]),
        "fftmech_diffusion_step": (i, [vp, vp, i, P(d), d, d, vp, d, vp, P(fftmech_solve_info)]),
        "fftmech_equilibrium_solve": (i, [vp, vp, vp, vp, P(d), vp, vp, vp, P(fftmech_solve_info)]),
        "fftmech_phasefield_solve": (i, [vp, vp, vp, vp, vp, vp, P(fftmech_solve_info)]),
        "fftmech_staggered_step": (i, [vp, P(fftmech_state), P(fftmech_step_params),
                                       P(fftmech_solve_info)]),
        "fftmech_staggered_step_async": (i, [vp, P(fftmech_state), P(fftmech_step_params)]),
        "fftmech_step_info": (i, [vp, P(fftmech_solve_info)]),
        "fftmech_adjoint_eigenstrain": (i, [vp, vp, vp, i, P(d), P(d), i, i, vp, P(d), P(fftmech_solve_info)]),
        "fftmech_autotune": (i, [vp, i, P(d), P(d), P(ctypes.c_char_p)]),
        "fftmech_set_launch_shapes": (i, [vp, ctypes.c_char_p]),
        "fftmech_problem_offset": (i, [vp, i, i, P(ctypes.c_longlong)]),
        "fftmech_graph_stats": (i, [vp, P(ctypes.c_longlong), P(ctypes.c_longlong), P(ctypes.c_longlong),
                                    P(i), P(ctypes.c_char_p)]),
        "fftmech_group_create": (i, [P(vp), P(vp), i, vp]),
        "fftmech_group_destroy": (i, [vp]),
        "fftmech_group_step": (i, [vp, P(P(fftmech_state)), P(P(fftmech_step_params)), P(P(fftmech_solve_info))]),
        "fftmech_group_stats": (i, [vp, P(ctypes.c_longlong), P(ctypes.c_longlong), P(ctypes.c_longlong)]),
        "fftmech_group_last_error": (ctypes.c_char_p, [vp]),
        "fftmech_staggered_step_many": (i, [P(vp), i, P(P(fftmech_state)), P(P(fftmech_step_params)),
                                            P(P(fftmech_solve_info))]),
        "fftmech_homogenise_operator": (i, [vp, vp, i, P(d), vp, vp, P(fftmech_solve_info)]),
        "fftmech_equilibrium_operator": (i, [vp, vp, vp, vp, P(d), i, vp, vp, P(fftmech_solve_info)]),
        "fftmech_phasefield_operator": (i, [vp, vp, vp, vp, i, vp, vp, P(fftmech_solve_info)]),
        "fftmech_bar_create": (i, [P(vp), vp, d, d, d, P(d)]),
        "fftmech_bar_destroy": (i, [vp]),
        "fftmech_bar_step": (i, [vp, P(fftmech_state), P(fftmech_step_params), P(fftmech_solve_info)]),
        "fftmech_bar_read": (i, [vp, P(d)]),
        "fftmech_bar_write": (i, [vp, P(d)]),
        "fftmech_fft": (i, [i, P(i), i, i, vp, vp]),
        "fftmech_fft_noalloc": (i, [i, P(i), i, i, vp, vp]),
        "fftmech_profile_enable": (i, [vp, i]),
        "fftmech_profile_read": (i, [vp, i, P(ctypes.c_longlong), P(d)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def ptr(x):
    """Address of a buffer: torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(rc, ctx=None, allow=(FFTMECH_OK,)):
    if rc in allow:
        return rc
    lib = load_library()
    msg = lib.fftmech_status_string(rc).decode()
    if ctx is not None:
        detail = lib.fftmech_last_error(ctx).decode()
        if detail:
            msg += ": " + detail
    raise FftmechError(rc, msg)


class FftmechError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fftmech status {status}: {msg}")
        self.status = status


# ---------------------------------------------------------------- same names as the C ABI

def fftmech_create(grid, mat, precision, opts, stream=None):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.fftmech_create(ctypes.byref(h), ctypes.byref(grid), ctypes.byref(mat), int(precision),
                            ctypes.byref(opts), stream)
    _check(rc)
    return h


def fftmech_create_batched(grid, batch, mat, precision, opts, stream=None):
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.fftmech_create_batched(ctypes.byref(h), ctypes.byref(grid), int(batch), ctypes.byref(mat),
                                    int(precision), ctypes.byref(opts), stream)
    _check(rc)
    return h


def fftmech_batch_size(ctx):
    return load_library().fftmech_batch_size(ctx)


def fftmech_destroy(ctx):
    return load_library().fftmech_destroy(ctx)


def fftmech_set_solver_opts(ctx, opts):
    return _check(load_library().fftmech_set_solver_opts(ctx, ctypes.byref(opts)), ctx)


def fftmech_status_string(status):
    return load_library().fftmech_status_string(int(status)).decode()


def fftmech_last_error(ctx):
    return load_library().fftmech_last_error(ctx).decode()


_SOLVER_OK = (FFTMECH_OK, FFTMECH_ERR_NOT_CONVERGED, FFTMECH_ERR_NONFINITE)


def _infos(ctx, per_problem):
    n = max(1, fftmech_batch_size(ctx)) * per_problem
    return (fftmech_solve_info * n)()


def _one_or_all(arr):
    return arr[0] if len(arr) == 1 else arr


def fftmech_diffusion_step(ctx, phase, mode, grad_c_mac, c_macro, dt, dirichlet_mask,
                           dirichlet_value, c, info=None):
    """Returns the solve record (a ctypes array of them for a batch)."""
    infos = _infos(ctx, 1)
    g = c_double3(*(list(grad_c_mac) + [0.0] * 3)[:3])
    rc = load_library().fftmech_diffusion_step(ctx, ptr(phase), int(mode), g, float(c_macro),
                                               float(dt), ptr(dirichlet_mask),
                                               float(dirichlet_value), ptr(c), infos)
    _check(rc, ctx, _SOLVER_OK)
    return _one_or_all(infos)


def fftmech_equilibrium_solve(ctx, phase, eig, damage, eps_mac, u, strain, stress, info=None):
    infos = _infos(ctx, 1)
    e = c_double6(*(list(eps_mac) + [0.0] * 6)[:6])
    rc = load_library().fftmech_equilibrium_solve(ctx, ptr(phase), ptr(eig), ptr(damage), e, ptr(u),
                                                  ptr(strain), ptr(stress), infos)
    _check(rc, ctx, _SOLVER_OK)
    return _one_or_all(infos)


def fftmech_phasefield_solve(ctx, strain, eig, phase, H, damage, info=None):
    infos = _infos(ctx, 1)
    rc = load_library().fftmech_phasefield_solve(ctx, ptr(strain), ptr(eig), ptr(phase), ptr(H),
                                                 ptr(damage), infos)
    _check(rc, ctx, _SOLVER_OK)
    return _one_or_all(infos)


def fftmech_staggered_step(ctx, state, params, infos=None):
    """Returns 3 records per problem: [diffusion, equilibrium, phase field]."""
    infos = infos or _infos(ctx, 3)
    rc = load_library().fftmech_staggered_step(ctx, ctypes.byref(state), ctypes.byref(params), infos)
    _check(rc, ctx, _SOLVER_OK)
    return infos


def fftmech_staggered_step_async(ctx, state, params):
    """Enqueues a staggered step (device pointers only) and returns at once."""
    rc = load_library().fftmech_staggered_step_async(ctx, ctypes.byref(state), ctypes.byref(params))
    _check(rc, ctx)
    return rc


def fftmech_step_info(ctx, infos=None):
    """Synchronises and returns the 3 records per problem of the last step."""
    infos = infos or _infos(ctx, 3)
    rc = load_library().fftmech_step_info(ctx, infos)
    _check(rc, ctx, _SOLVER_OK)
    return infos


def fftmech_adjoint_eigenstrain(ctx, phase, e_field, ramp, eps_mac, objective, checkpoint_every, grad):
    """Objective value J of the staggered solve with the eigenstrain
    ramp[s] e(x) and its gradient dJ/de written to `grad` (device buffers);
    returns (J, the 3 records of the forward's last step)."""
    steps = len(ramp)
    r = (ctypes.c_double * steps)(*[float(x) for x in ramp])
    e = c_double6(*(list(eps_mac or []) + [0.0] * 6)[:6])
    J = ctypes.c_double(0.0)
    infos = (fftmech_solve_info * 3)()
    rc = load_library().fftmech_adjoint_eigenstrain(ctx, ptr(phase), ptr(e_field), steps, r, e, int(objective),
                                                    int(checkpoint_every), ptr(grad), ctypes.byref(J), infos)
    _check(rc, ctx, _SOLVER_OK)
    return J.value, infos


def fftmech_autotune(ctx, iterations=30):
    """Tunes the context's launch shapes; returns (us per iteration before,
    after, description of the chosen shapes)."""
    b, a = ctypes.c_double(0), ctypes.c_double(0)
    desc = ctypes.c_char_p()
    _check(load_library().fftmech_autotune(ctx, int(iterations), ctypes.byref(b), ctypes.byref(a),
                                           ctypes.byref(desc)), ctx)
    return b.value, a.value, (desc.value or b"").decode()


def fftmech_set_launch_shapes(ctx, shapes):
    """Applies launch shapes given as fftmech_autotune's description."""
    _check(load_library().fftmech_set_launch_shapes(ctx, shapes.encode()), ctx)


def fftmech_problem_offset(ctx, problem, components):
    off = ctypes.c_longlong(0)
    _check(load_library().fftmech_problem_offset(ctx, int(problem), int(components), ctypes.byref(off)), ctx)
    return off.value


def fftmech_graph_stats(ctx):
    """(graphs built, graph launches, kernels run by the replays, disabled, reason)."""
    b = ctypes.c_longlong(0)
    n = ctypes.c_longlong(0)
    k = ctypes.c_longlong(0)
    dis = ctypes.c_int(0)
    why = ctypes.c_char_p()
    _check(load_library().fftmech_graph_stats(ctx, ctypes.byref(b), ctypes.byref(n), ctypes.byref(k),
                                              ctypes.byref(dis), ctypes.byref(why)), ctx)
    return b.value, n.value, k.value, dis.value, (why.value or b"").decode()


def fftmech_fft(ndim, n, precision, inverse, data, stream=None):
    nn = c_int3(*(list(n) + [1, 1, 1])[:3])
    rc = load_library().fftmech_fft(int(ndim), nn, int(precision), int(inverse), ptr(data), stream)
    _check(rc)
    return rc


FFTMECH_FFT_NOALLOC_MAX_N = 2187


def fftmech_fft_noalloc(ndim, n, precision, inverse, data, stream=None):
    """Same transform as fftmech_fft without any device allocation (twiddles
    in a fixed array inside the library; sizes up to FFTMECH_FFT_NOALLOC_MAX_N)."""
    nn = c_int3(*(list(n) + [1, 1, 1])[:3])
    rc = load_library().fftmech_fft_noalloc(int(ndim), nn, int(precision), int(inverse), ptr(data),
                                            stream)
    _check(rc)
    return rc


def fftmech_staggered_step_many(ctxs, states, params, infos=None):
    """Staggered steps of several contexts concurrently; returns the list of
    per-context info arrays (3 records per problem)."""
    n = len(ctxs)
    infos = infos or [_infos(c, 3) for c in ctxs]
    c_arr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    s_arr = (ctypes.POINTER(fftmech_state) * n)(*[ctypes.pointer(s) for s in states])
    p_arr = (ctypes.POINTER(fftmech_step_params) * n)(*[ctypes.pointer(p) for p in params])
    i_arr = (ctypes.POINTER(fftmech_solve_info) * n)(*[ctypes.cast(x, ctypes.POINTER(fftmech_solve_info))
                                                       for x in infos])
    rc = load_library().fftmech_staggered_step_many(c_arr, n, s_arr, p_arr, i_arr)
    _check(rc, None, _SOLVER_OK)
    return infos


def _handles(ctxs):
    n = len(ctxs)
    return (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])


def fftmech_group_create(ctxs, stream=None):
    h = ctypes.c_void_p()
    _check(load_library().fftmech_group_create(ctypes.byref(h), _handles(ctxs), len(ctxs), stream))
    return h


def fftmech_group_destroy(group):
    return load_library().fftmech_group_destroy(group)


def fftmech_group_step(group, ctxs, states, params, infos=None):
    """One staggered step of every context of the group (one graph launch);
    returns the per-context info arrays (3 records per problem)."""
    n = len(states)
    infos = infos or [_infos(c, 3) for c in ctxs]
    s_arr = (ctypes.POINTER(fftmech_state) * n)(*[ctypes.pointer(s) for s in states])
    p_arr = (ctypes.POINTER(fftmech_step_params) * n)(*[ctypes.pointer(p) for p in params])
    i_arr = (ctypes.POINTER(fftmech_solve_info) * n)(*[ctypes.cast(x, ctypes.POINTER(fftmech_solve_info))
                                                       for x in infos])
    lib = load_library()
    rc = lib.fftmech_group_step(group, s_arr, p_arr, i_arr)
    if rc not in _SOLVER_OK:
        raise FftmechError(rc, lib.fftmech_status_string(rc).decode() + ": " +
                           lib.fftmech_group_last_error(group).decode())
    return infos


def fftmech_group_last_error(group):
    return load_library().fftmech_group_last_error(group).decode()


def fftmech_group_stats(group):
    """(graphs built, graph launches, kernels run)."""
    b, n, k = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(load_library().fftmech_group_stats(group, ctypes.byref(b), ctypes.byref(n), ctypes.byref(k)))
    return b.value, n.value, k.value


def fftmech_homogenise_operator(ctx, phase, gradient, grad_c_mac, phi=None, grad_c=None):
    """Homogenised diffusion with the gradient operator `gradient`
    (FFTMECH_GRAD_*); device buffers; returns the solve record."""
    info = fftmech_solve_info()
    g = c_double3(*(list(grad_c_mac) + [0.0] * 3)[:3])
    rc = load_library().fftmech_homogenise_operator(ctx, ptr(phase), int(gradient), g, ptr(phi), ptr(grad_c),
                                                    ctypes.byref(info))
    _check(rc, ctx, _SOLVER_OK)
    return info


def fftmech_equilibrium_operator(ctx, phase, eig, damage, eps_mac, gradient, strain=None, stress=None):
    """Equilibrium with the gradient operator `gradient` (FFTMECH_GRAD_*);
    device buffers (eig, damage double or None); returns the solve record."""
    info = fftmech_solve_info()
    e = c_double6(*(list(eps_mac) + [0.0] * 6)[:6])
    rc = load_library().fftmech_equilibrium_operator(ctx, ptr(phase), ptr(eig), ptr(damage), e, int(gradient),
                                                     ptr(strain), ptr(stress), ctypes.byref(info))
    _check(rc, ctx, _SOLVER_OK)
    return info


def fftmech_phasefield_operator(ctx, phase, strain, eig, gradient, H, d):
    """History update and phase field with the gradient operator `gradient`
    (FFTMECH_GRAD_*); device buffers (double); returns the solve record."""
    info = fftmech_solve_info()
    rc = load_library().fftmech_phasefield_operator(ctx, ptr(phase), ptr(strain), ptr(eig), int(gradient), ptr(H),
                                                    ptr(d), ctypes.byref(info))
    _check(rc, ctx, _SOLVER_OK)
    return info


def fftmech_bar_create(ctx, length, dt, flux_in, c0=None):
    """Macroscale bar over the RVEs of a batched context (Sec. 3.2)."""
    h = ctypes.c_void_p()
    arr = None
    if c0 is not None:
        arr = (ctypes.c_double * len(c0))(*[float(x) for x in c0])
    _check(load_library().fftmech_bar_create(ctypes.byref(h), ctx, float(length), float(dt), float(flux_in), arr), ctx)
    return h


def fftmech_bar_destroy(bar):
    return load_library().fftmech_bar_destroy(bar)


def fftmech_bar_step(bar, ctx, state, params):
    """One macro time step (one staggered step of every RVE); returns the
    3 records per RVE."""
    infos = _infos(ctx, 3)
    rc = load_library().fftmech_bar_step(bar, ctypes.byref(state), ctypes.byref(params), infos)
    _check(rc, ctx, _SOLVER_OK)
    return infos


def fftmech_bar_read(bar, n):
    out = (ctypes.c_double * n)()
    _check(load_library().fftmech_bar_read(bar, out))
    return list(out)


def fftmech_bar_write(bar, values):
    arr = (ctypes.c_double * len(values))(*[float(x) for x in values])
    _check(load_library().fftmech_bar_write(bar, arr))


class Group:
    """Owns one fftmech group of contexts (create / destroy)."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        self.handle = fftmech_group_create([c.handle for c in self.contexts], stream)

    def step(self, states, params):
        return fftmech_group_step(self.handle, [c.handle for c in self.contexts], states, params)

    def stats(self):
        return fftmech_group_stats(self.handle)

    def close(self):
        if self.handle:
            fftmech_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fftmech_profile_enable(ctx, enable):
    return _check(load_library().fftmech_profile_enable(ctx, int(enable)), ctx)


def fftmech_profile_read(ctx, kclass):
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(load_library().fftmech_profile_read(ctx, int(kclass), ctypes.byref(n), ctypes.byref(ms)), ctx)
    return n.value, ms.value


# ---------------------------------------------------------------- small conveniences

def make_grid(shape, h, h_diff=1.0):
    """shape in array order (ny, nx) or (nz, ny, nx)."""
    g = fftmech_grid()
    g.dim = len(shape)
    n = list(reversed(shape)) + [1] * (3 - len(shape))
    g.n = c_int3(*n)
    g.h = h
    g.h_diff = h_diff
    return g


def make_materials(m):
    """From any object with the fftmech_materials field names as attributes."""
    out = fftmech_materials()
    for k, _ in fftmech_materials._fields_:
        setattr(out, k, float(getattr(m, k)))
    return out


def make_opts(tol=1e-8, max_iter=20000, replace_residual=1, check_every=16, launch_mode=0,
              execution=FFTMECH_EXEC_GRAPH, precond=FFTMECH_PRECOND_LAPLACE):
    o = fftmech_solver_opts()
    o.tol = tol
    o.max_iter = max_iter
    o.replace_residual = replace_residual
    o.check_every = check_every
    o.launch_mode = launch_mode
    o.execution = execution
    o.precond = precond
    return o


class Context:
    """Owns one fftmech context (create / destroy)."""

    def __init__(self, shape, materials, precision=FFTMECH_FP64, h=5e-6, h_diff=1.0,
                 tol=1e-8, max_iter=20000, replace_residual=1, check_every=16, stream=None, batch=1,
                 launch_mode=0, execution=FFTMECH_EXEC_GRAPH, precond=FFTMECH_PRECOND_LAPLACE):
        self.shape = tuple(shape)
        self.precision = precision
        self.batch = batch
        self.grid = make_grid(shape, h, h_diff)
        self.mat = make_materials(materials)
        self.opts = make_opts(tol, max_iter, replace_residual, check_every, launch_mode, execution, precond)
        if batch == 1:
            self.handle = fftmech_create(self.grid, self.mat, precision, self.opts, stream)
        else:
            self.handle = fftmech_create_batched(self.grid, batch, self.mat, precision, self.opts, stream)

    @property
    def field_dtype(self):
        return np.float64 if self.precision == FFTMECH_FP64 else np.float32

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        fftmech_set_solver_opts(self.handle, self.opts)

    def close(self):
        if self.handle:
            fftmech_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
