"""The reference-medium preconditioner of the equilibrium PCG
(fftmech_solver_opts.precond = FFTMECH_PRECOND_REFERENCE; 2D column pass,
3D z pass), through the C ABI:

- a homogeneous medium of the solid's Poisson ratio with a random
  eigenstrain converges in one iteration on the FP64 path (the
  preconditioner is the exact inverse there: a sign, conjugate or
  mirror-column slip breaks that), where the Laplace preconditioner needs
  many; the mixed path's float recursion also stops after one iteration,
  its FP64 true residual then sits at float storage level (~1e-7) above
  tol = 1e-8, and each restart from it takes one more exact iteration;
- random carpets (odd and even sizes: the self-mirrored columns kx = 0 and
  nx / 2 and rows ky = ny / 2; the deferred and the last-block reductions;
  a batch): the strain matches the FP64 oracle (FP64 within 1e-10, mixed
  within 1e-5) in fewer iterations than with the Laplace preconditioner;
- graph and host-driven execution agree bit for bit;
- 3D (the z pass pairs the line sets ky and ny - ky and the columns kx and
  nx - kx, with the half spectrum of u_z): the homogeneous medium in one
  FP64 iteration on odd and even sizes (self-mirrored kx = nx / 2, ky =
  ny / 2, kz = nz / 2), sponges and tiled 2 x 2 sponges against the oracle
  in fewer iterations than the Laplace preconditioner, a batch, and graph
  against host-driven execution.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from microstructures import random_carpet, random_sponge
from microstructures.workloads import Materials
from oracle import elasticity
from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

pytestmark = pytest.mark.gpu

H = 5e-6
MAT = Materials()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    fm.load_library()


def solve(phases, e, prec, precond, tol, execution=fm.FFTMECH_EXEC_GRAPH):
    B = len(phases)
    shape = phases[0].shape
    N = phases[0].size
    d = len(shape)
    nv = 3 if d == 2 else 6
    ctx = fm.Context(shape, MAT, prec, h=H, tol=tol, max_iter=20000, batch=B, precond=precond,
                     execution=execution)
    ft = torch.float64 if prec == fm.FFTMECH_FP64 else torch.float32
    ph = torch.as_tensor(np.concatenate([p.ravel() for p in phases])).cuda()
    eig = torch.as_tensor(np.concatenate([x.ravel() for x in e])).to(ft).cuda()
    u = torch.zeros(d * N * B, dtype=torch.float64, device="cuda")
    strain = torch.zeros(nv * N * B, dtype=ft, device="cuda")
    infos = fm.fftmech_equilibrium_solve(ctx.handle, ph, eig, None, [0] * 6, u, strain, None)
    infos = [infos] if B == 1 else list(infos)
    ctx.close()
    return strain.double().cpu().numpy().reshape(B, nv, *shape), [i.iters for i in infos], [i.status for i in infos]


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def carpet(shape, seed):
    """A random 3x3 carpet, or 2x2 carpets tiled along x for other sizes."""
    ny, nx = shape
    if ny == nx and ny % 3 == 0:
        return random_carpet(ny, 0.30, seed)[0]
    return np.tile(random_carpet(ny, 0.30, seed, base=2)[0], (1, nx // ny))


def pore_eig(phase, seed):
    rng = np.random.default_rng(seed)
    return np.where(phase == 0, 1e-3 * (1 + 0.2 * rng.standard_normal(phase.shape)), 0.0)


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
@pytest.mark.parametrize("shape", [(81, 81), (64, 96)])
def test_homogeneous_medium_converges_in_one_iteration(shape, prec):
    ph = np.ones(shape, dtype=np.uint8)
    e = 1e-3 * np.random.default_rng(3).standard_normal(shape)
    tol = 1e-12 if prec == fm.FFTMECH_FP64 else 1e-8
    _, it_ms, st = solve([ph], [e], prec, fm.FFTMECH_PRECOND_REFERENCE, tol)
    _, it_lp, _ = solve([ph], [e], prec, fm.FFTMECH_PRECOND_LAPLACE, tol)
    print("homogeneous", shape, prec, "iterations reference", it_ms, "laplace", it_lp)
    assert st == [fm.FFTMECH_OK]
    assert it_ms[0] == (1 if prec == fm.FFTMECH_FP64 else 3) and it_lp[0] >= 10


@pytest.mark.parametrize("prec,tol,bound", [(fm.FFTMECH_FP64, 1e-12, 1e-10), (fm.FFTMECH_MIXED, 1e-8, 1e-5)])
@pytest.mark.parametrize("shape,seeds", [((81, 81), [41]), ((128, 256), [42]), ((243, 243), [43, 44, 45])])
def test_carpets_match_oracle_in_fewer_iterations(shape, seeds, prec, tol, bound):
    phases = [carpet(shape, s) for s in seeds]
    e = [pore_eig(p, 7 + i) for i, p in enumerate(phases)]
    got, it_ms, st = solve(phases, e, prec, fm.FFTMECH_PRECOND_REFERENCE, tol)
    _, it_lp, _ = solve(phases, e, prec, fm.FFTMECH_PRECOND_LAPLACE, tol)
    assert all(s == fm.FFTMECH_OK for s in st)
    for b, ph in enumerate(phases):
        ref = elasticity.equilibrium_solve(ph, e[b], np.ones(ph.shape), [0, 0, 0], MAT, H, tol=1e-12)
        err = rel(got[b], ref["strain"])
        print("carpet", shape, b, prec, "iterations reference", it_ms[b], "laplace", it_lp[b], "strain rel", err)
        assert err < bound, err
        assert it_ms[b] < it_lp[b]


def test_large_batch_last_block_form_and_execution_modes():
    # 40 x 243^2 = 2.4 M voxels per launch: the last-block reductions
    phases = [random_carpet(243, 0.30, 100 + s)[0] for s in range(40)]
    e = [pore_eig(p, 200 + s) for s, p in enumerate(phases)]
    a, it_a, st = solve(phases, e, fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_REFERENCE, 1e-8)
    b, it_b, _ = solve(phases, e, fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_REFERENCE, 1e-8,
                       execution=fm.FFTMECH_EXEC_HOST)
    assert all(s == fm.FFTMECH_OK for s in st)
    assert it_a == it_b and np.array_equal(a, b)
    for k in (0, 39):
        ref = elasticity.equilibrium_solve(phases[k], e[k], np.ones(phases[k].shape), [0, 0, 0], MAT, H, tol=1e-12)
        assert rel(a[k], ref["strain"]) < 1e-5


# ---------------------------------------------------------------- 3D

def sponge(shape, seed):
    """A random 3x3 sponge, one tiled along z (nz a multiple of ny = nx, a
    power of 3), or a 2x2 one tiled along x for other sizes."""
    nz, ny, nx = shape
    if nz == ny == nx and nx % 3 == 0:
        return random_sponge(nx, 0.35, seed)[0]
    if ny == nx and nx % 3 == 0 and nz % nx == 0:
        return np.ascontiguousarray(np.tile(random_sponge(nx, 0.35, seed)[0], (nz // nx, 1, 1)))
    return np.ascontiguousarray(np.tile(random_carpet(ny, 0.35, seed, base=2, dim=3)[0], (1, 1, nx // ny)))


@pytest.mark.parametrize("prec", [fm.FFTMECH_FP64, fm.FFTMECH_MIXED])
@pytest.mark.parametrize("shape", [(9, 8, 6), (6, 9, 8), (27, 27, 27)])
def test_homogeneous_medium_converges_in_one_iteration_3d(shape, prec):
    ph = np.ones(shape, dtype=np.uint8)
    e = 1e-3 * np.random.default_rng(4).standard_normal(shape)
    tol = 1e-12 if prec == fm.FFTMECH_FP64 else 1e-8
    _, it_ms, st = solve([ph], [e], prec, fm.FFTMECH_PRECOND_REFERENCE, tol)
    _, it_lp, _ = solve([ph], [e], prec, fm.FFTMECH_PRECOND_LAPLACE, tol)
    print("homogeneous 3d", shape, prec, "iterations reference", it_ms, "laplace", it_lp)
    assert st == [fm.FFTMECH_OK]
    assert it_ms[0] == (1 if prec == fm.FFTMECH_FP64 else 3) and it_lp[0] >= 10


@pytest.mark.parametrize("prec,tol,bound", [(fm.FFTMECH_FP64, 1e-12, 1e-10), (fm.FFTMECH_MIXED, 1e-8, 1e-5)])
@pytest.mark.parametrize("shape,seeds", [((27, 27, 27), [51]), ((16, 16, 32), [52]), ((27, 27, 27), [53, 54]),
                                         ((81, 27, 27), [55]), ((243, 9, 9), [56])])
def test_sponges_match_oracle_in_fewer_iterations(shape, seeds, prec, tol, bound):
    """nz = 81 and 243 take the compile-time z plans on the mixed path."""
    phases = [sponge(shape, s) for s in seeds]
    e = [pore_eig(p, 17 + i) for i, p in enumerate(phases)]
    got, it_ms, st = solve(phases, e, prec, fm.FFTMECH_PRECOND_REFERENCE, tol)
    _, it_lp, _ = solve(phases, e, prec, fm.FFTMECH_PRECOND_LAPLACE, tol)
    assert all(s == fm.FFTMECH_OK for s in st)
    for b, ph in enumerate(phases):
        ref = elasticity.equilibrium_solve(ph, e[b], np.ones(ph.shape), [0] * 6, MAT, H, tol=1e-12)
        err = rel(got[b], ref["strain"])
        print("sponge", shape, b, prec, "iterations reference", it_ms[b], "laplace", it_lp[b], "strain rel", err)
        assert err < bound, err
        assert it_ms[b] < it_lp[b]


def test_graph_and_host_driven_agree_3d():
    phases = [sponge((27, 27, 27), 60 + s) for s in range(2)]
    e = [pore_eig(p, 70 + s) for s, p in enumerate(phases)]
    a, it_a, st = solve(phases, e, fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_REFERENCE, 1e-8)
    b, it_b, _ = solve(phases, e, fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_REFERENCE, 1e-8,
                       execution=fm.FFTMECH_EXEC_HOST)
    assert all(s == fm.FFTMECH_OK for s in st)
    assert it_a == it_b and np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(729, 729), (243, 243, 243)])
def test_full_size_reference_medium_and_laplace_agree(shape):
    """At the benchmark sizes (729^2 carpet, 243^3 sponge; mixed, tol 1e-8)
    the two preconditioners are independent routes to the same solution:
    the strain fields agree within the solver tolerance's reach, and the
    reference medium takes fewer iterations."""
    seed = 81
    ph = carpet(shape, seed) if len(shape) == 2 else sponge(shape, seed)
    e = pore_eig(ph, seed + 1)
    a, it_ms, st = solve([ph], [e], fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_REFERENCE, 1e-8)
    b, it_lp, st2 = solve([ph], [e], fm.FFTMECH_MIXED, fm.FFTMECH_PRECOND_LAPLACE, 1e-8)
    err = rel(a, b)
    print("full size", shape, "iterations reference", it_ms, "laplace", it_lp, "strain rel", err)
    assert st == [fm.FFTMECH_OK] and st2 == [fm.FFTMECH_OK]
    assert err < 1e-5 and it_ms[0] < it_lp[0]
