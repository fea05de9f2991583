"""CUDA path against the FP64 CPU oracle at the grid sizes the product runs
through its compile-time FFT plans (lines of 256, 512, 1024 and 2187 points
in the x-line and the column passes), on launches large enough to take the
last-block reduction form (more than 2^21 voxels per launch, 2D and 3D), and
over all ten steps of the Sierpinski workload (81 x 81, homogenised
diffusion, prescribed pore eigenstrain, Algorithm 1).

Tolerances (relative L2 over all voxels and components unless stated): FP64
GPU path within 1e-10 of the oracle (both solved to a 1e-12 relative
residual); mixed path within 1e-5 on strain and stress, 1e-6 on the
concentration and 1e-4 max-abs on damage.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials, left_face_mask, sierpinski_static
from oracle import elasticity, phasefield, staggered
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT_DMG = Materials(E_pore=2e9, M_ppt=2.2)  # stiff pores and a large molar volume: damage develops


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    if nb == 0:
        return float(np.linalg.norm(np.ravel(a)))
    return float(np.linalg.norm(np.ravel(a - b)) / nb)


def ftype(prec):
    return torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32


def cropped_carpet(shape, seed):
    n = max(shape)
    base = 2 if n & (n - 1) == 0 else 3
    ph, _ = random_carpet(n, 0.30, seed, base=base)
    return np.ascontiguousarray(ph[:shape[0], :shape[1]])


def gpu_steps(phase, prec, steps, params_fn, tol, mat, batch=1):
    """Runs `steps` staggered steps on device buffers; params_fn(step) gives
    the fftmech_step_params. phase: (B, ...) for a batch."""
    shape = phase.shape[1:] if batch > 1 else phase.shape
    N = int(np.prod(shape))
    dim = len(shape)
    nv = 3 if dim == 2 else 6
    ft = ftype(prec)
    ctx = fm.Context(shape, mat, prec, h=H, h_diff=1.0, tol=tol, batch=batch, max_iter=20000)
    B = batch
    bufs = {k: torch.zeros(m * N * B, dtype=dt, device="cuda") for k, m, dt in
            [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", dim, torch.float64),
             ("strain", nv, ft), ("stress", nv, ft), ("H", 1, ft), ("damage", 1, torch.float64)]}
    bufs["phase"] = torch.as_tensor(np.ascontiguousarray(phase).ravel()).cuda()
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    infos = []
    keep = []
    for s in range(steps):
        p, k = params_fn(s)
        keep.append(k)
        infos.append(fm.fftmech_staggered_step(ctx.handle, st, p))
    torch.cuda.synchronize()
    out = {k: v.double().cpu().numpy() for k, v in bufs.items()}
    ctx.close()
    return out, infos


def transient_params(mask_np, dt):
    mask = torch.as_tensor(np.ascontiguousarray(mask_np).ravel()).cuda()

    def fn(_s):
        p = fm.fftmech_step_params()
        p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
        p.dt = dt
        p.dirichlet_mask = mask.data_ptr()
        p.dirichlet_value = 1.0
        p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
        return p, mask
    return fn


def check_fields(out, ref, shape, prec, b=None, what=""):
    N = int(np.prod(shape))
    nv = 3 if len(shape) == 2 else 6

    def view(k, m):
        v = out[k]
        if b is not None:
            v = v[b * m * N:(b + 1) * m * N]
        return v.reshape(((m,) if m > 1 else ()) + tuple(shape))

    c, strain, stress = view("c", 1), view("strain", nv), view("stress", nv)
    d, Hh = view("damage", 1), view("H", 1)
    errs = {"c": rel(c, ref["c"]), "strain": rel(strain, ref["strain"]), "stress": rel(stress, ref["stress"]),
            "d_maxabs": float(np.abs(d - ref["d"]).max())}
    if np.linalg.norm(ref["d"]) > 0:
        errs["d"] = rel(d, ref["d"])
    if np.linalg.norm(ref["H"]) > 0:
        errs["H"] = rel(Hh, ref["H"])
    print(what, shape, "FP64" if prec == fm.FFTMECH_FP64 else "MIXED", errs)
    if prec == fm.FFTMECH_FP64:
        for k in ("c", "strain", "stress", "d", "H"):
            if k in errs:
                assert errs[k] < 1e-10, (k, errs[k])
    else:
        assert errs["c"] < 1e-6
        assert errs["strain"] < 1e-5 and errs["stress"] < 1e-5
        assert errs["d_maxabs"] < 1e-4


# ---------------------------------------------------------------- compile-time plans

# (shape, seed): seeds whose cropped carpet puts pores next to the source, so
# that the step precipitates and the equilibrium has a load
PLAN_SHAPES = [((27, 1024), 41), ((1024, 27), 41), ((16, 512), 42), ((512, 16), 41), ((27, 256), 41),
               ((256, 27), 41), ((9, 2187), 41), ((2187, 9), 41)]


@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
@pytest.mark.parametrize("shape,seed", PLAN_SHAPES, ids=[f"{a}x{b}" for (a, b), _ in PLAN_SHAPES])
def test_staggered_step_through_line_plans(shape, seed, prec):
    """One transient staggered step (diffusion, precipitation, equilibrium,
    history, phase field) on a grid whose long side takes a compile-time
    plan, against the oracle. The long transient steps (dt = (nx/4)^2 / 10)
    are stiff: the FP64 path is solved to 1e-13 so that its distance to the
    oracle (solved to 1e-12) stays below 1e-10. FP64 contexts with x lines of
    2187 points do not fit the FP64 residual kernel's shared memory and are
    rejected as an unsupported size."""
    phase = cropped_carpet(shape, seed)
    if prec == fm.FFTMECH_FP64 and shape[1] == 2187:
        with pytest.raises(fm.FftmechError) as ei:
            fm.Context(shape, MAT_DMG, prec, h=H)
        assert ei.value.status == fm.FFTMECH_ERR_UNSUPPORTED_SIZE
        return
    mask = left_face_mask(phase)
    dt = (shape[1] / 4.0) ** 2 / 10
    ref = staggered.step(staggered.initial_state(phase), phase, MAT_DMG, H, 1.0, staggered.DIFF_TRANSIENT,
                         staggered.EIG_FROM_PRECIPITATE, dt=dt, mask=mask, c_dirichlet=1.0, tol=1e-12)[0]
    tol = 1e-13 if prec == fm.FFTMECH_FP64 else 1e-10
    out, infos = gpu_steps(phase, prec, 1, transient_params(mask, dt), tol, MAT_DMG)
    assert all(i.status == fm.FFTMECH_OK for i in infos[0])
    assert ref["eig"].max() > 0
    check_fields(out, ref, shape, prec, what="plans")


# ---------------------------------------------------------------- last-block forms

def test_2d_batch_above_2pow21_voxels_matches_oracle():
    """36 carpets of 243^2 (2.13 M voxels per launch: last-block reductions),
    FP64, one transient staggered step; problems 0, 17 and 35 against the
    oracle."""
    n, B = 243, 36
    phases = np.stack([random_carpet(n, 0.30, 100 + b)[0] for b in range(B)])
    masks = np.stack([left_face_mask(p) for p in phases])
    dt = (n / 4.0) ** 2 / 10
    out, infos = gpu_steps(phases, fm.FFTMECH_FP64, 1, transient_params(masks, dt), 1e-12, MAT_DMG, batch=B)
    assert all(i.status == fm.FFTMECH_OK for i in infos[0])
    for b in (0, 17, 35):
        ref = staggered.step(staggered.initial_state(phases[b]), phases[b], MAT_DMG, H, 1.0,
                             staggered.DIFF_TRANSIENT, staggered.EIG_FROM_PRECIPITATE, dt=dt, mask=masks[b],
                             c_dirichlet=1.0, tol=1e-12)[0]
        check_fields(out, ref, (n, n), fm.FFTMECH_FP64, b=b, what=f"2D batch problem {b}")


@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
def test_3d_batch_above_2pow21_voxels_matches_oracle(prec):
    """128 sponges of 27^3 (2.52 M voxels per launch: last-block reductions
    in every 3D kernel), pore eigenstrain, no diffusion, one staggered
    step; problems 0, 63 and 127 against the oracle."""
    n, B = 27, 128
    phases = np.stack([random_sponge(n, 0.35, 500 + b)[0] for b in range(B)])
    eigs = np.where(phases == 0, 2e-2, 0.0)
    ef = torch.as_tensor(eigs.ravel()).to(ftype(prec)).cuda()

    def params(_s):
        p = fm.fftmech_step_params()
        p.diffusion_mode = fm.FFTMECH_DIFF_NONE
        p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
        p.eig_field = ef.data_ptr()
        p.eig_scale = 1.0
        return p, ef

    tol = 1e-12 if prec == fm.FFTMECH_FP64 else 1e-10
    out, infos = gpu_steps(phases, prec, 1, params, tol, MAT_DMG, batch=B)
    assert all(i.status == fm.FFTMECH_OK for i in infos[0])
    for b in (0, 63, 127):
        ref = staggered.step(staggered.initial_state(phases[b]), phases[b], MAT_DMG, H, 1.0,
                             staggered.DIFF_NONE, staggered.EIG_PRESCRIBED, eig_field=eigs[b], tol=1e-12)[0]
        assert ref["d"].max() > 1e-3
        check_fields(out, ref, (n, n, n), prec, b=b, what=f"3D batch problem {b}")


# ---------------------------------------------------------------- Sierpinski, all ten steps

def test_sierpinski_workload_all_ten_steps_fp64():
    """The Sierpinski workload exactly as benchmarked (81 x 81, pores at
    1e-3 of the solid stiffness, pore eigenstrain 1e-3, homogenised
    diffusion with grad c_mac = (1, 0) and c(X) = 1), all ten staggered
    steps in FP64, every step against the oracle."""
    w = sierpinski_static()
    phase = w.phase
    ef = torch.as_tensor(w.eig.ravel()).cuda()

    def params(s):
        p = fm.fftmech_step_params()
        p.diffusion_mode = fm.FFTMECH_DIFF_HOMOGENISE
        p.grad_c_mac = fm.c_double3(*w.grad_c_mac)
        p.c_macro = w.c_macro
        p.eig_mode = fm.FFTMECH_EIG_PRESCRIBED
        p.eig_field = ef.data_ptr()
        p.eig_scale = w.eig_ramp[s]
        return p, ef

    shape = phase.shape
    N = phase.size
    ctx = fm.Context(shape, w.materials, fm.FFTMECH_FP64, h=w.h, h_diff=w.h_diff, tol=1e-12)
    bufs = {k: torch.zeros(m * N, dtype=torch.float64, device="cuda") for k, m in
            [("c", 1), ("c_ppt", 1), ("eig", 1), ("u", 2), ("strain", 3), ("stress", 3), ("H", 1), ("damage", 1)]}
    bufs["phase"] = torch.as_tensor(phase.ravel()).cuda()
    st = fm.fftmech_state()
    for k, v in bufs.items():
        setattr(st, k, v.data_ptr())
    ref = staggered.initial_state(phase)
    for s in range(w.steps):
        ref, rinfo = staggered.step(ref, phase, w.materials, w.h, w.h_diff, staggered.DIFF_HOMOGENISE,
                                    staggered.EIG_PRESCRIBED, eig_field=w.eig, eig_scale=w.eig_ramp[s],
                                    grad_c_mac=w.grad_c_mac[:2], c_macro=w.c_macro, tol=1e-12)
        p, _k = params(s)
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        assert all(i.status == fm.FFTMECH_OK for i in infos)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in bufs.items()}
        check_fields(out, ref, shape, fm.FFTMECH_FP64, what=f"sierpinski step {s}")
        en = elasticity.elastic_energy(ref["strain"], ref["stress"], ref["eig"], w.h)
        assert infos[1].elastic_energy == pytest.approx(en, rel=1e-10)
        assert infos[2].total_damage == pytest.approx(ref["d"].sum(), rel=1e-10, abs=1e-300)
    ctx.close()
