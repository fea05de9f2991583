"""Launch modes of the PCG iteration.

- Programmatic dependent launches (bit 0 clear, the default) against plain
  stream order: every kernel waits on the device for its predecessor, so
  both must give bit-identical fields and the same iteration counts. A
  missing wait would show up here as a race (a field that differs between
  the modes or from run to run).
- The fused direction-stencil kernel of latency-bound 2D grids (bit 1
  set) against the split direction and stencil kernels (the default):
  the same operator and direction, so a fixed number of iterations gives
  the same iterate up to the rounding of the <p, K p> summation order
  (FP64: 1e-12), on grids whose rows do not divide evenly into the fused
  kernel's blocks, with a Dirichlet mask; whole staggered steps agree to
  the solver tolerance.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials, left_face_mask
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT = Materials(E_pore=2e9, M_ppt=2.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def transient_state(phases, prec, dt):
    n = phases[0].size
    d = phases[0].ndim
    nv = 3 if d == 2 else 6
    B = len(phases)
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    spec = [("c", 1, torch.float64), ("c_ppt", 1, ft), ("eig", 1, ft), ("u", d, torch.float64),
            ("strain", nv, ft), ("stress", nv, ft), ("H", 1, ft), ("damage", 1, torch.float64)]
    bufs = {k: torch.zeros(m * n * B, dtype=t, device="cuda") for k, m, t in spec}
    bufs["phase"] = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
    bufs["mask"] = torch.as_tensor(np.concatenate([left_face_mask(p).ravel() for p in phases])).cuda()
    st = fm.fftmech_state()
    for k in ("phase", "c", "c_ppt", "eig", "u", "strain", "stress", "H", "damage"):
        setattr(st, k, bufs[k].data_ptr())
    p = fm.fftmech_step_params()
    p.diffusion_mode = fm.FFTMECH_DIFF_TRANSIENT
    p.dt = dt
    p.dirichlet_mask = bufs["mask"].data_ptr()
    p.dirichlet_value = 1.0
    p.eig_mode = fm.FFTMECH_EIG_FROM_PRECIPITATE
    return bufs, st, p


def run_steps(phases, prec, launch_mode, steps=2, tol=1e-8):
    shape = phases[0].shape
    n = min(shape)
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=tol, batch=len(phases), launch_mode=launch_mode)
    bufs, st, p = transient_state(phases, prec, (n / 4.0) ** 2 / 10)
    iters = []
    for _ in range(steps):
        infos = fm.fftmech_staggered_step(ctx.handle, st, p)
        k = len(phases) * 3
        assert all(infos[i].status == fm.FFTMECH_OK for i in range(k))
        iters.append([infos[i].iters for i in range(k)])
    torch.cuda.synchronize()
    ctx.close()
    return {k: bufs[k].cpu().numpy() for k in ("c", "u", "strain", "stress", "damage")}, iters


@pytest.mark.parametrize("fuse", [0, 2])
@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
@pytest.mark.parametrize("n,seeds", [(81, (7, 8)), (243, (9,))])
def test_dependent_launches_bit_identical_2d(prec, n, seeds, fuse):
    phases = [random_carpet(n, 0.30, s)[0] for s in seeds]
    a, ia = run_steps(phases, prec, 0 + fuse)
    b, ib = run_steps(phases, prec, 1 + fuse)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert a["damage"].max() > 0


def test_dependent_launches_bit_identical_3d():
    phases = [np.ascontiguousarray(random_sponge(27, 0.35, s)[0]) for s in (3, 4)]
    a, ia = run_steps(phases, fm.FFTMECH_MIXED, 0, steps=1)
    b, ib = run_steps(phases, fm.FFTMECH_MIXED, 1, steps=1)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_dependent_launches_repeatable():
    """Two runs in the default mode agree bit for bit (deterministic
    reductions; no read of a buffer that a still-running kernel writes)."""
    phases = [random_carpet(81, 0.30, s)[0] for s in (11, 12, 13)]
    a, ia = run_steps(phases, fm.FFTMECH_MIXED, 0)
    b, ib = run_steps(phases, fm.FFTMECH_MIXED, 0)
    assert ia == ib
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


GRIDS = [((729, 729), (21,)), ((243, 96), tuple(range(22, 30))), ((48, 81), (30,))]


def cut_carpets(shape, seeds):
    ny, nx = shape
    return [np.ascontiguousarray(random_carpet(max(shape), 0.30, s)[0][:ny, :nx]) for s in seeds]


def k_iterations(phases, prec, launch_mode, kind, k=12, shapes=None):
    """The first k PCG iterations (tol 0) of a transient diffusion step with
    a Dirichlet face (D = 1) or of an equilibrium solve with a pore
    eigenstrain (D = 2): no residual replacement happens before the 16th.
    shapes: launch shapes to apply first (fftmech_set_launch_shapes)."""
    shape = phases[0].shape
    B, N = len(phases), phases[0].size
    ctx = fm.Context(shape, MAT, prec, h=H, h_diff=1.0, tol=0.0, max_iter=k, batch=B, launch_mode=launch_mode)
    if shapes:
        fm.fftmech_set_launch_shapes(ctx.handle, shapes)
    ph = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
    rng = np.random.default_rng(5)
    if kind == "diffusion":
        mask = torch.as_tensor(np.concatenate([left_face_mask(p).ravel() for p in phases])).cuda()
        c = torch.as_tensor(rng.random(B * N)).cuda()
        fm.fftmech_diffusion_step(ctx.handle, ph, fm.FFTMECH_DIFF_TRANSIENT, [0.0, 0.0], 0.0, 20.0, mask, 1.0, c)
        out = c
    else:
        ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
        eig = torch.where(ph == 0, 1e-3, 0.0).to(ft)
        out = torch.zeros(2 * B * N, dtype=torch.float64, device="cuda")
        fm.fftmech_equilibrium_solve(ctx.handle, ph, eig, None, [0.0] * 6, out, None, None)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("kind", ["diffusion", "equilibrium"])
@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
@pytest.mark.parametrize("shape,seeds", GRIDS)
def test_fused_direction_stencil_iterate_for_iterate(prec, shape, seeds, kind):
    """The host's rule gives 729 rows blocks of three own rows, a batch of
    eight 243 x 96 grids blocks of seven ending with a five-row block, and
    48 x 81 one row per block. Every grid has blocks whose halo rows wrap
    around the periodic boundary. A wrong halo row or a misplaced q would
    move the iterate at O(1)."""
    phases = cut_carpets(shape, seeds)
    a = k_iterations(phases, prec, 0, kind)
    b = k_iterations(phases, prec, 2, kind)
    e = rel(a, b)
    print(kind, shape, e)
    assert e < (1e-12 if prec == fm.FFTMECH_FP64 else 1e-5), e


@pytest.mark.parametrize("prec", [fm.FFTMECH_MIXED, fm.FFTMECH_FP64])
@pytest.mark.parametrize("shape,seeds", GRIDS)
def test_fused_direction_stencil_matches_split(prec, shape, seeds):
    """Whole staggered steps (tol 1e-8). The summation order moves the
    iterates by rounding; over hundreds of iterations of the ill-conditioned
    diffusion solve, CG's loss of orthogonality turns that into a path a
    few iterations longer or shorter (the float recursion of the mixed
    path more so), ending at the same tolerance."""
    phases = cut_carpets(shape, seeds)
    a, ia = run_steps(phases, prec, 0)
    b, ib = run_steps(phases, prec, 2)
    print("iterations fused", ia, "split", ib)
    fp64 = prec == fm.FFTMECH_FP64
    for step_a, step_b in zip(ia, ib):
        for x, y in zip(step_a, step_b):
            assert abs(x - y) <= 3 + (0.03 if fp64 else 0.1) * y, (ia, ib)
    for k in a:
        e = rel(a[k], b[k])
        print(k, e)
        assert e < 1e-5, (k, e)
    assert a["damage"].max() > 0


@pytest.mark.parametrize("kind", ["diffusion", "equilibrium"])
@pytest.mark.parametrize("shapes", ["cols=2", "cols=8", "cols=2 L_ds=1", "cols=8 L_ds=2", "L_ds=4",
                                    "L_dir=3 L_upd=1 ty=8 grid=300"])
def test_launch_shapes_729(shapes, kind):
    """Launch shapes that the autotuner may pick (applied through
    fftmech_set_launch_shapes): every column strip width of the compile-time
    729-point plan, fused kernels of one, two and four rows (the last two
    ending with a one-row block), other line and stencil
    shapes. Twelve iterations agree with the rule-based shapes to the
    rounding of the reductions' block partitions (mixed path)."""
    phases = cut_carpets((729, 729), (41,))
    a = k_iterations(phases, fm.FFTMECH_MIXED, 0, kind)
    b = k_iterations(phases, fm.FFTMECH_MIXED, 0, kind, shapes=shapes)
    e = rel(b, a)
    print(shapes, kind, e)
    assert e < 1e-5, e


def test_launch_shapes_round_trip_and_errors():
    ctx = fm.Context((243, 243), MAT, fm.FFTMECH_MIXED, h=H)
    fm.fftmech_set_launch_shapes(ctx.handle, "cols=2 L_ds=3")
    _, _, desc = fm.fftmech_autotune(ctx.handle, 0)
    assert "cols=2" in desc and "L_ds=3" in desc
    fm.fftmech_set_launch_shapes(ctx.handle, desc + " (cached)")
    for bad in ("cols=3", "L_ds=-1", "ty=5", "foo=1", "cols"):
        with pytest.raises(RuntimeError):
            fm.fftmech_set_launch_shapes(ctx.handle, bad)
    assert fm.fftmech_autotune(ctx.handle, 0)[2] == desc
    ctx.close()
